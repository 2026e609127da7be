// solve.cu -- the contact solve of one substep (Eq. (7)-(8)) by the
// quasi-Newton iteration of Alg. 1 (Sec. IV-C, V-B), entirely on the device.
//
// One cooperative launch runs the whole iteration. The participating thread
// blocks (as many as the contact count needs, at most one per SM) step
// through the phases in lockstep, separated by a grid barrier whose spin has
// an iteration limit (on expiry the kernel records MPM_ERR_TIMEOUT and every
// block returns). Only the nodes in the stencil of some contact can change
// (everywhere else the gradient M (v - v*) is zero at v = v*), so the node
// phases run over a contact-node list built at the start; the momentum norm
// adds the grid update's sum of m |v*|^2 over the other nodes.
//
// Per iteration:
//   G  contacts: v_c = J v + b + alpha J dv (a compensated gather of the
//      double-float iterate); gradient (3) and Hessian (3x3) of the lagged contact
//      potential, scattered with weights w and w^2 (the 3x3 diagonal blocks of
//      J^T (d2 l_c) J, Eq. (10)).
//   N  contact nodes: v += alpha dv (double-float, into the other buffer of
//      the iterate), g = M (v - v*) + J^T dl_c (Eq. (9)), H = M + contact
//      blocks, stopping norms, dv = -H^-1 g by 3x3 Cholesky; grid sums of the
//      line search, A = dv^T M dv and B = dv^T M (v - v*).
//   C  contacts: dv_c = J dv.
//   L  exact line search (Alg. 1): f'(alpha) = B + alpha A + sum_p dl_c . dv_c
//      is monotone (f convex); each pass evaluates it at 8 points in one
//      contact sweep: first on a geometric grid (0, 4^-5 .. 4) to bracket the
//      root, then at the Newton and secant estimates and points that split
//      the bracket, until |f'| <= ls_rel_tol |f'(0)|. Up to kLocalLsMax contacts every block
//      runs the whole line search by itself over all contacts (their v_c and
//      dv_c sit in L2), so its passes need no grid barrier; above that the
//      contacts are split over the blocks and each pass ends in a grid-wide
//      reduction.
// Every block reads the same reduced sums (or computes the same ones in the
// same order), so all take the same decisions. Scalar sums are accumulated
// per thread and per warp in FP32, across warps and blocks as double-float
// (hi, lo) pairs with error-free FP32 transforms: GB300's FP64 pipe is narrow
// enough that FP64 on these serial paths costs more than the rest of a pass.
#include <cfloat>

#include "kernels.h"

namespace mpmcr {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kContactsPerBlock = 128;  // forward solve: 8 contacts per warp in the gather phases
constexpr int kAdjContactsPerBlock = 16;  // adjoint: one contact per warp
constexpr int kLocalLsMax = 4096;      // up to this many contacts each block line-searches alone
constexpr int kLsPoints = 8;
constexpr int kRedWidth = 16;              // (hi, lo) pairs per block and reduction
constexpr int kMaxSolveBlocks = 256;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a barrier gives up after 1 s
constexpr unsigned kSpinCap = 1u << 28;  // backstop on the number of polls

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

struct Barrier {
  unsigned* bar;  // arrival counters (kBarWords, zeroed between launches)
  unsigned n;     // the participating blocks
  uint32_t* status;
  int* poison;    // set on expiry: the next solve first clears the node scratch
  int cluster;    // nonzero: the blocks are one thread-block cluster
  unsigned extra; // arrivals awaited that never come (barrier time-limit test only)
  unsigned blk;   // this block's index among the participating blocks
};

// Barrier of all threads of the thread-block cluster (hardware barrier; the
// arrive releases and the wait acquires every thread's earlier memory
// operations at cluster scope, global reductions included).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// (hi, lo) pair at the same shared-memory offset in block `rank` of the cluster
__device__ __forceinline__ float2 ld_cluster_f2(const float2* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(ra)
               : "memory");
  return v;
}

// Device-wide barrier of the participating blocks on one 64-bit arrival
// counter that only grows: the k-th barrier is complete when it reaches
// (k + 1) x blocks, which each block reads off its own ticket, so nothing is
// reset or published by the last arriver. (A single counter measured faster
// on GB300 than counters per group of 16 blocks: 1.3 against 2.1 us per
// barrier of 152 blocks.) Thread 0 publishes its block's writes (fence),
// arrives, and polls with a time limit (1 s of the global timer); on expiry
// it returns false (the caller then returns; the other blocks expire at the
// same or their next barrier). A single participating block needs only
// __syncthreads; the blocks of one cluster use the cluster barrier.
__device__ bool grid_sync(Barrier& B) {
  if (B.cluster) {
    cluster_sync_all();
    return true;
  }
  __syncthreads();
  if (B.n == 1 && B.extra == 0) return true;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned long long* top = reinterpret_cast<unsigned long long*>(B.bar);
    const unsigned long long per = (unsigned long long)B.n + B.extra;
    __threadfence();
    const unsigned long long ticket = atomicAdd(top, 1ull);
    const unsigned long long target = (ticket / per + 1ull) * per;
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire(top) < target) {
      ++spins;
      if (((spins & 63u) == 0u && global_ns() - t0 > kWaitLimitNs) || spins > kSpinCap) {
        atomicOr(B.status, kStTimeout);
        if (B.poison) atomicExch(B.poison, 1);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// double-float value (hi, lo), |lo| <= ulp(hi) / 2
__device__ __forceinline__ float2 df_norm(float S, float E) {
  const float hi = S + E;
  return make_float2(hi, E - (hi - S));
}

// (S, E) += (hi, lo)
__device__ __forceinline__ void df_acc(float& S, float& E, float2 x) {
  float s, e;
  two_sum(S, x.x, s, e);
  S = s;
  E += e + x.y;
}

// Block sums of NV per-thread values, exchanged through per-block slots and
// summed by every block in the same fixed order (deterministic). Returns the
// double-float totals in s_tot (shared) and false if the barrier expired.
// `part`: the global slot of a device-wide reduction; in a cluster the block
// sums go to the shared-memory slot `cpart` instead and every block reads the
// others' through distributed shared memory.
template <int NV>
__device__ bool reduce_all(const float (&v)[NV], float2* part, Barrier& B, float (*s_red)[kRedWidth],
                           float2* s_tot, float2* cpart = nullptr) {
  static_assert(NV <= kWarps && NV <= kRedWidth, "one warp per reduced value");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if constexpr (NV == 16) {
    // reduce-scatter butterfly: after the exchange over lane bit b each lane
    // keeps half of its values (those whose index bit b equals its lane bit
    // b), so lane l ends with value l & 15 summed over the warp (16 shuffles
    // instead of 80)
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = v[i];
#pragma unroll
    for (int b = 0, m = 8; b < 4; ++b, m >>= 1) {
      const bool hi = (lane >> b) & 1;
#pragma unroll
      for (int j = 0; j < m; ++j) {
        const float keep = hi ? x[2 * j + 1] : x[2 * j];
        const float send = hi ? x[2 * j] : x[2 * j + 1];
        x[j] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << b);
      }
    }
    const float t = x[0] + __shfl_xor_sync(0xffffffffu, x[0], 16);
    if (lane < 16) s_red[w][lane] = t;
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      float x = v[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) s_red[w][i] = x;
    }
  }
  __syncthreads();
  // block sum of value w: lane l < kWarps holds warp l's, a butterfly over
  // those lanes (compensated)
  if (w < NV) {
    float S = lane < kWarps ? s_red[lane][w] : 0.f, E = 0.f;
#pragma unroll
    for (int o = kWarps / 2; o > 0; o >>= 1) {
      const float S2 = __shfl_xor_sync(0xffffffffu, S, o);
      const float E2 = __shfl_xor_sync(0xffffffffu, E, o);
      float s2, e;
      two_sum(S, S2, s2, e);
      S = s2;
      E = E + E2 + e;
    }
    if (lane == 0) {
      if (B.cluster)
        cpart[w] = df_norm(S, E);
      else if (B.n == 1)
        s_tot[w] = df_norm(S, E);
      else
        part[w * kMaxSolveBlocks + B.blk] = df_norm(S, E);
    }
  }
  if (!grid_sync(B)) return false;
  if (B.cluster || B.n > 1) {
    // warp i sums value i over the blocks: lane l takes blocks l, l + 32, ...
    // (their loads in flight together), then a butterfly over the warp's
    // double-float pairs; the same fixed order in every block
    if (w < NV) {
      float S = 0.f, E = 0.f;
      if (B.cluster) {
        if (lane < (int)B.n) {
          const float2 t = ld_cluster_f2(cpart + w, (unsigned)lane);
          S = t.x;
          E = t.y;
        }
      } else {
        for (int b0 = 0; b0 < (int)B.n; b0 += 8 * 32) {
          float2 t[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int b = b0 + 32 * u + lane;
            t[u] = b < (int)B.n ? __ldcg(part + w * kMaxSolveBlocks + b) : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) df_acc(S, E, t[u]);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float S2 = __shfl_xor_sync(0xffffffffu, S, o);
        const float E2 = __shfl_xor_sync(0xffffffffu, E, o);
        float s2, e;
        two_sum(S, S2, s2, e);
        S = s2;
        E = E + E2 + e;
      }
      if (lane == 0) s_tot[w] = df_norm(S, E);
    }
    __syncthreads();
  }
  return true;
}

// Warp-cooperative stencil access: lane l < 27 owns node (l % 3, l / 3 % 3, l / 9)
// of the contact's 3x3x3 stencil, so the 27 loads or reductions of a contact
// go out together instead of in register-limited groups.
struct LaneNode {
  int node;
  float w;
};

__device__ __forceinline__ LaneNode lane_node(const GridDev& g, const float4& xp, int lane) {
  Stencil s;
  stencil(g, xp.x, xp.y, xp.z, s);
  const int l = lane < 27 ? lane : 0;
  const int cx = l % 3, cy = (l / 3) % 3, cz = l / 9;
  LaneNode r;
  r.node = node_index(g, s.base[0] + cx, s.base[1] + cy, s.base[2] + cz);
  r.w = lane < 27 ? s.w[0][cx] * s.w[1][cy] * s.w[2][cz] : 0.f;
  return r;
}

// Contact groups of the forward solve's gather / scatter phases: kGrp lanes
// per contact, lane sub of a group owning stencil nodes sub, sub + kGrp, ...
constexpr int kGrp = 4;
constexpr int kGrpPerWarp = 32 / kGrp;
constexpr int kGrpNodes = (27 + kGrp - 1) / kGrp;

struct GroupNodes {
  int node[kGrpNodes];
  float w[kGrpNodes];
};

__device__ __forceinline__ void group_nodes(const GridDev& g, const float4& xp, int sub,
                                            GroupNodes& r) {
  Stencil s;
  stencil(g, xp.x, xp.y, xp.z, s);
#pragma unroll
  for (int j = 0; j < kGrpNodes; ++j) {
    const int c = sub + kGrp * j;
    const int cc = c < 27 ? c : 26;
    const int cx = cc % 3, cy = (cc / 3) % 3, cz = cc / 9;
    r.node[j] = node_index(g, s.base[0] + cx, s.base[1] + cy, s.base[2] + cz);
    r.w[j] = c < 27 ? s.w[0][cx] * s.w[1][cy] * s.w[2][cz] : 0.f;
  }
}

// compensated sum of (S, E) pairs over the lanes of a group, bitwise the same
// in each of them (TwoSum's error term is exact whichever operand comes first)
__device__ __forceinline__ float group_comp_sum(float S, float E) {
#pragma unroll
  for (int o = 1; o < kGrp; o <<= 1) {
    const float S2 = __shfl_xor_sync(0xffffffffu, S, o);
    const float E2 = __shfl_xor_sync(0xffffffffu, E, o);
    float s2, e;
    two_sum(S, S2, s2, e);
    S = s2;
    E = E + E2 + e;
  }
  return S + E;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ void load_contact(const Contacts& C, int p, float4& xp, float (&n)[3],
                                             float& n0) {
  xp = C.xp[p];
  const float4 q = C.nrm[p];
  n[0] = q.x; n[1] = q.y; n[2] = q.z;
  n0 = q.w;
}

// Line-search cache: a thread's k-th contact (k < kLsCacheDepth) keeps its
// line form in shared-memory slot k * kThreads + tid across the passes of one
// line search, packed into three float4: (v_n, e_n, vhat, phi0),
// (mu n0, body, v_t.x, v_t.y), (v_t.z, e_t); k and d come from the body table.
constexpr int kLsCacheDepth = 4;
constexpr int kLsCacheSlots = kLsCacheDepth * kThreads;

__device__ __forceinline__ void line_store(float4* cache, int slot, const ContactLine& L, int body) {
  cache[3 * slot] = make_float4(L.vn0, L.en, L.vhat, L.phi0);
  cache[3 * slot + 1] = make_float4(L.mun0, __int_as_float(body), L.vt[0], L.vt[1]);
  cache[3 * slot + 2] = make_float4(L.vt[2], L.et[0], L.et[1], L.et[2]);
}

__device__ __forceinline__ void line_load(const float4* cache, int slot, const DevBody* bodies,
                                          float h, float eps2, ContactLine& L) {
  const float4 q0 = cache[3 * slot], q1 = cache[3 * slot + 1], q2 = cache[3 * slot + 2];
  const DevBody& bd = bodies[__float_as_int(q1.y)];
  L.vn0 = q0.x; L.en = q0.y; L.vhat = q0.z; L.phi0 = q0.w;
  L.mun0 = q1.x; L.vt[0] = q1.z; L.vt[1] = q1.w; L.vt[2] = q2.x;
  L.et[0] = q2.y; L.et[1] = q2.z; L.et[2] = q2.w;
  L.hk = h * bd.k;
  L.h = h;
  L.d = bd.d;
  L.eps2 = eps2;
  L.et2 = L.et[0] * L.et[0] + L.et[1] * L.et[1] + L.et[2] * L.et[2];
}

// Exact line search of Alg. 1 on f'(alpha) = B + alpha A + sum_p dl_c . dv_c,
// which is continuous and non-decreasing (f convex). Each pass has f' and f''
// at 8 points; the bracket [lo, hi] keeps f'(lo) < 0 <= f'(hi). The first
// pass is 0 and a geometric grid (ratio 4, extended while f' < 0); later
// passes evaluate the Newton step from the best point, the secant of the
// bracket and six points that split it (geometrically while it spans more
// than a factor 4, else its thirds and points around the Newton step).
// Stops when |f'(best)| <= rel_tol |f'(0)|. Run by the 32 lanes of warp 0:
// lane l owns point l & 7; the bracket and the best point (kept alike in
// every lane) are updated by butterfly reductions over the 8 points.
struct LineSearch {
  enum { kMore = 0, kDone = 1, kFailed = 2 };
  float lo, hi, flo, fhi, best, fbest, f2best, f0;
  bool have_f0;
  float pt;  // this lane's point
  __device__ void reset() {
    const int k = threadIdx.x & (kLsPoints - 1);
    lo = 0.f; hi = -1.f; flo = fhi = best = fbest = f2best = f0 = 0.f;
    have_f0 = false;
    // first pass: 0 and a geometric grid 4^-5 .. 4 (quasi-Newton steps on
    // stiff contacts are often much shorter than 1)
    pt = k == 0 ? 0.f : exp2f(2.0f * (float)(k - 6));
  }
  // f' = B + alpha A + S is formed in double-float (its terms can cancel);
  // the bracket logic runs in FP32 (alpha is applied in FP32 anyway)
  __device__ int update(const float2* tot, float2 A, float2 B, float rel_tol, bool last) {
    const int k = threadIdx.x & (kLsPoints - 1);
    const float x = pt;
    CompSum c;
    c.S = B.x;
    c.E = B.y + x * A.y + tot[k].y;
    c.add_prod(x, A.x);
    c.add(tot[k].x);
    const float d = c.value();
    const float d2 = (A.x + tot[kLsPoints + k].x) + (A.y + tot[kLsPoints + k].y);
    if (!have_f0) {  // the first pass's point 0 is alpha = 0
      f0 = __shfl_sync(0xffffffffu, d, 0);
      flo = f0;
      best = 0.f;
      fbest = f0;
      f2best = __shfl_sync(0xffffffffu, d2, 0);
      have_f0 = true;
    }
    // candidates of this pass: the largest point with f' < 0 (ties: the later
    // point), the smallest with f' >= 0 (ties: the earlier), the smallest
    // |f'| (ties: the earlier)
    float clo = d < 0.f ? x : -1.f, cflo = d;
    int klo = k;
    float chi = d < 0.f ? INFINITY : x, cfhi = d;
    int khi = k;
    float cb = fabsf(d), cbx = x, cbd = d, cbd2 = d2;
    int kb = k;
#pragma unroll
    for (int o = 1; o < kLsPoints; o <<= 1) {
      const float olo = __shfl_xor_sync(0xffffffffu, clo, o);
      const float oflo = __shfl_xor_sync(0xffffffffu, cflo, o);
      const int oklo = __shfl_xor_sync(0xffffffffu, klo, o);
      if (olo > clo || (olo == clo && oklo > klo)) { clo = olo; cflo = oflo; klo = oklo; }
      const float ohi = __shfl_xor_sync(0xffffffffu, chi, o);
      const float ofhi = __shfl_xor_sync(0xffffffffu, cfhi, o);
      const int okhi = __shfl_xor_sync(0xffffffffu, khi, o);
      if (ohi < chi || (ohi == chi && okhi < khi)) { chi = ohi; cfhi = ofhi; khi = okhi; }
      const float ob = __shfl_xor_sync(0xffffffffu, cb, o);
      const float obx = __shfl_xor_sync(0xffffffffu, cbx, o);
      const float obd = __shfl_xor_sync(0xffffffffu, cbd, o);
      const float obd2 = __shfl_xor_sync(0xffffffffu, cbd2, o);
      const int okb = __shfl_xor_sync(0xffffffffu, kb, o);
      if (ob < cb || (ob == cb && okb < kb)) { cb = ob; cbx = obx; cbd = obd; cbd2 = obd2; kb = okb; }
    }
    if (clo >= lo) { lo = clo; flo = cflo; }
    if (chi != INFINITY && (hi < 0.f || chi < hi)) { hi = chi; fhi = cfhi; }
    if (cb < fabsf(fbest)) { best = cbx; fbest = cbd; f2best = cbd2; }
    if (!(f0 < 0.f)) { best = 0.f; return kDone; }  // no descent left at working precision
    if (fabsf(fbest) <= rel_tol * fabsf(f0) || last) return kDone;
    if (hi < 0.f) {  // root beyond the grid: keep growing by 4x
      if (lo >= 1024.f) { best = lo; return kFailed; }
      pt = lo * (float)(4 << (2 * k));
      return kMore;
    }
    if (hi - lo <= 1e-7f * hi) return kDone;
    const float w = hi - lo;
    float xn = f2best > 0.f ? best - fbest / f2best : 0.5f * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
    float xs = lo - flo * w / (fhi - flo);
    if (!(xs > lo && xs < hi)) xs = 0.5f * (lo + hi);
    // a bracket spanning more than a factor 4 (or reaching down to 0) is
    // split geometrically; a narrow one by its thirds (the bracket shrinks at
    // least threefold) and points 1% and 10% of its width either side of
    // the Newton point (where the root lies once Newton converges)
    if (k == 0) {
      pt = xn;
    } else if (k == 1) {
      pt = xs;
    } else {
      const float lo_g = lo > 0.f ? lo : hi * (1.0f / 4096.0f);
      if (hi > 4.f * lo_g) {
        const float r = exp2f(__log2f(hi / lo_g) / 7.0f);
        float xg = lo_g;
        for (int j = 2; j <= k; ++j) xg *= r;
        pt = xg;
      } else {
        const float cw = k == 2 ? 1.f / 3.f : k == 3 ? 2.f / 3.f : k == 4 ? -0.1f
                         : k == 5 ? 0.1f : k == 6 ? -0.01f : 0.01f;
        float xc = k < 4 ? lo + cw * w : xn + cw * w;
        if (!(xc > lo && xc < hi)) xc = lo + (float)(k - 1) / 7.0f * w;
        pt = xc;
      }
    }
    return kMore;
  }
};

// kCluster: the solve of up to a.cluster_max contacts by the blocks of one
// thread-block cluster (hardware cluster barriers, block sums exchanged
// through distributed shared memory); otherwise the cooperative launch over
// as many blocks as the contacts need, for more contacts than that. `block`
// is this block's index among the `grid_blocks` blocks of the solve (a
// batched launch gives every scene one block of its own).
template <bool kCluster>
__device__ __forceinline__ void solve_body(const SolveArgs& a, int block, int grid_blocks) {
  __shared__ DevBody s_body[kMaxBodies];
  __shared__ float2 s_cpart[4][kRedWidth];  // cluster: block sums, a ring of four reductions
  __shared__ float s_red[kWarps][kRedWidth];
  __shared__ float2 s_tot[kRedWidth];
  __shared__ float s_imp[kMaxBodies][6];
  __shared__ float s_pts[kLsPoints];
  __shared__ float2 s_A, s_B;
  __shared__ float s_alpha;
  __shared__ int s_dec;
  extern __shared__ float4 s_line[];  // 3 x kLsCacheSlots: the line-search cache (+ stencils)
  LineSearch ls;  // used by warp 0
  const int tid = threadIdx.x;
  const int count = *a.C.count;
  const int nc = count < a.C.cap ? count : a.C.cap;
  if (nc == 0) return;  // v = v* already (set by the grid update)
  // (every block of a launch reads the same count: the choice is uniform)
  if (kCluster ? nc > a.cluster_max : nc <= a.cluster_max) return;  // the other kernel's
  int nblk = grid_blocks;  // a cluster: all of its blocks
  if (!kCluster) {
    nblk = (nc + kContactsPerBlock - 1) / kContactsPerBlock;
    nblk = nblk < grid_blocks ? nblk : grid_blocks;
    nblk = nblk < kMaxSolveBlocks ? nblk : kMaxSolveBlocks;
    if (block >= nblk) return;  // not needed for this many contacts
  }

  for (int i = tid; i < a.nb * (int)(sizeof(DevBody) / 4); i += kThreads)
    reinterpret_cast<float*>(s_body)[i] = reinterpret_cast<const float*>(a.bodies)[i];
  for (int i = tid; i < kMaxBodies * 6; i += kThreads) (&s_imp[0][0])[i] = 0.f;
  __syncthreads();

  // phase timers (block 0, thread 0): list, G, N, line search, impulses
  unsigned long long tph[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
  unsigned long long tmark = global_ns();
  auto lap = [&](int ph) {
    if (block == 0 && tid == 0) {
      const unsigned long long now = global_ns();
      tph[ph] += now - tmark;
      tmark = now;
    }
  };
  // (wait_extra > 0 only in the test of the barrier's time limit: the
  // barrier then waits for arrivals that never come)
  Barrier B{a.bar, (unsigned)nblk, a.status, a.poison, kCluster ? 1 : 0,
            kCluster ? 0u : (unsigned)a.wait_extra, (unsigned)block};
  const int gtid = block * kThreads + tid;
  const int gstride = nblk * kThreads;
  const int lane = tid & 31;
  const int gwarp = gtid >> 5;
  const int nwarps = gstride >> 5;
  const GridDev& g = a.g;
  // per-block partial sums, a ring of 4 slots of kMaxSolveBlocks x kRedWidth;
  // a slot is rewritten two reductions later, after every block has read it
  int rslot = 0;
  auto next_slot = [&]() -> float2* {
    float2* s = reinterpret_cast<float2*>(a.red) + (size_t)(rslot & 3) * kMaxSolveBlocks * kRedWidth;
    ++rslot;
    return s;
  };
  // in a cluster the block sums go to a ring of shared-memory slots instead
  // (rewritten four reductions later, after every block has read it)
  int cslot = 0;
  auto next_cpart = [&]() -> float2* { return kCluster ? s_cpart[(cslot++) & 3] : nullptr; };

  // a solve that gave up at a barrier left node flags and gradient
  // accumulators behind: clear them over the whole grid first
  if (__ldcg(a.poison)) {
    const size_t n_nodes = (size_t)storage_nodes(g);
    for (size_t t = gtid; t < n_nodes; t += gstride) {
      a.G.cflag[t] = 0;
      a.G.acc0[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.G.acc1[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.G.acc2[t] = 0.f;
    }
    if (!grid_sync(B)) return;
    if (gtid == 0) *a.poison = 0;
  }

  // ---- contact-node list: the union of the contacts' stencils (a thread
  // per contact; the warp takes its list slots with one atomic)
  for (int p0 = gtid & ~31; p0 < nc; p0 += gstride) {
    const int p = p0 + lane;
    int node[27];
    unsigned won = 0u;  // 27 bits: this thread claimed the node first
    if (p < nc) {
      const float4 xp = a.C.xp[p];
      Stencil s;
      stencil(g, xp.x, xp.y, xp.z, s);
#pragma unroll
      for (int c = 0; c < 27; ++c) {
        node[c] = node_index(g, s.base[0] + c % 3, s.base[1] + (c / 3) % 3, s.base[2] + c / 9);
        if (atomicExch(a.G.cflag + node[c], 1) == 0) won |= 1u << c;
      }
    }
    const int cnt = __popc(won);
    int incl = cnt;  // inclusive prefix sum over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int slot0 = 0;
    if (lane == 31 && incl > 0) slot0 = atomicAdd(a.G.n_cnodes, incl);
    int slot = __shfl_sync(0xffffffffu, slot0, 31) + incl - cnt;
    if (won) {
#pragma unroll
      for (int c = 0; c < 27; ++c)
        if ((won >> c) & 1u) {
          if (slot < a.G.cnodes_cap) a.G.cnodes[slot] = node[c];
          ++slot;
        }
    }
  }
  if (!grid_sync(B)) return;
  lap(0);
  int ncn = __ldcg(a.G.n_cnodes);
  ncn = ncn < a.G.cnodes_cap ? ncn : a.G.cnodes_cap;
  // sum of m |v*|^2 over the grid (FP64 from the grid update) as double-float
  const double pstar2_d = __ldcg(a.G.pstar2);
  const float pstar2_hi = (float)pstar2_d, pstar2_lo = (float)(pstar2_d - (double)pstar2_hi);
  const float eps_a = (float)a.eps_a, eps_r = (float)a.eps_r;

  // The iterate v = hi + lo is double buffered: in phase G every contact node
  // writes v_next = v_cur + alpha dv while every contact gathers
  // v_c = J v_cur + b + alpha J dv from the untouched v_cur. Gathering v_c
  // afresh keeps it equal to J v (an incrementally updated v_c drifts from
  // J v over thousands of FP32 updates).
  float4* vcur = a.G.v;
  float4* vnxt = a.G.v2;
  float4* lcur = a.G.vlo;
  float4* lnxt = a.G.vlo2;
  // Gather / scatter phases: kGrp lanes per contact (lane group grp of the
  // warp, lane sub of the group owns stencil nodes sub, sub + kGrp, ...), so
  // a warp works on kGrpPerWarp contacts at once. The contacts of a warp's
  // first round stay in registers across the iterations.
  const int grp = lane / kGrp, sub = lane % kGrp;
  const int wfirst = gwarp * kGrpPerWarp;
  const int rstride = nwarps * kGrpPerWarp;
  const int own_p = wfirst + grp;
  const bool own = own_p < nc;
  // (the stencil of that contact in shared memory, beside the line-search
  // cache: registers are kept for the gathers in flight)
  int* s_own_node = reinterpret_cast<int*>(s_line + 3 * kLsCacheSlots) + tid * kGrpNodes;
  float* s_own_w = reinterpret_cast<float*>(s_line + 3 * kLsCacheSlots) + kThreads * kGrpNodes +
                   tid * kGrpNodes;
  {
    GroupNodes gn;
    group_nodes(g, own ? a.C.xp[own_p] : make_float4(0.f, 0.f, 0.f, 0.f), sub, gn);
#pragma unroll
    for (int j = 0; j < kGrpNodes; ++j) {
      s_own_node[j] = gn.node[j];
      s_own_w[j] = gn.w[j];
    }
  }
  auto own_nodes = [&](GroupNodes& gn) {
#pragma unroll
    for (int j = 0; j < kGrpNodes; ++j) {
      gn.node[j] = s_own_node[j];
      gn.w[j] = s_own_w[j];
    }
  };
  // this thread's first contact node (the list is fixed for the solve)
  const int my_node = gtid < ncn ? a.G.cnodes[gtid] : -1;
  // line search alone in each block (no grid barrier) or split over blocks
  const bool local_ls = kCluster ? nc <= kThreads : nc <= kLocalLsMax;
  const int ls_first = local_ls ? tid : gtid, ls_stride = local_ls ? kThreads : gstride;
  Barrier Bl{nullptr, 1u, a.status, nullptr, 0, 0u, 0u};
  const float eps2 = a.eps_s * a.eps_s;
  float alpha = 0.f;
  int it = 0, ls_passes = 0;
  float resid = 0.f;
  for (;;) {
    // ---- G: step by alpha, contact gradient / Hessian blocks (kGrp lanes per
    // contact)
    const float al = alpha;
    auto phase_g = [&](int p, bool valid, const float4& xp, const float (&n)[3], float n0,
                       const float4& bb, int body, const GroupNodes& gn) {
      const float4 dvc = valid && it > 0 ? __ldcg(a.C.dvc + p) : make_float4(0.f, 0.f, 0.f, 0.f);
      float u[3];
      {
        // compensated v_c = J v over the group's nodes: exact products w*hi
        // as (p, pe), plus w*lo
        float S[3] = {0.f, 0.f, 0.f}, E[3] = {0.f, 0.f, 0.f};
        if (valid) {
          // all of the group's loads first, so that they are in flight together
          float4 hq[kGrpNodes], lq[kGrpNodes];
#pragma unroll
          for (int j = 0; j < kGrpNodes; ++j) {
            if (sub + kGrp * j >= 27) continue;
            hq[j] = __ldcg(vcur + gn.node[j]);
            lq[j] = __ldcg(lcur + gn.node[j]);
          }
#pragma unroll
          for (int j = 0; j < kGrpNodes; ++j) {
            if (sub + kGrp * j >= 27) continue;
            const float4 h = hq[j], l = lq[j];
            const float w = gn.w[j];
            const float hv[3] = {h.x, h.y, h.z}, lv[3] = {l.x, l.y, l.z};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float pr = w * hv[c];
              const float pe = fmaf(w, hv[c], -pr) + w * lv[c];
              float t, e;
              two_sum(S[c], pr, t, e);
              S[c] = t;
              E[c] += e + pe;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = group_comp_sum(S[c], E[c]);
      }
      if (!valid) return;
      {
        // + b + alpha J dv, compensated (the same in every lane of the group)
        const float bv[3] = {bb.x, bb.y, bb.z}, dv3[3] = {dvc.x, dvc.y, dvc.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          CompSum cs;
          cs.S = u[c];
          cs.add(bv[c]);
          cs.add_prod(al, dv3[c]);
          u[c] = cs.value();
        }
      }
      if (sub == 0) a.C.vc[p] = make_float4(u[0], u[1], u[2], 0.f);
      const DevBody& bd = s_body[body];
      ContactLaw L;
      contact_law(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u, L);
      float gr[3], H[6];
      contact_grad(L, n, gr);
      contact_hess(L, n, H);
#pragma unroll
      for (int j = 0; j < kGrpNodes; ++j) {
        if (sub + kGrp * j >= 27) continue;
        const float w = gn.w[j], w2 = w * w;
        red_add_v4(a.G.acc0 + gn.node[j], w * gr[0], w * gr[1], w * gr[2], w2 * H[0]);
        red_add_v4(a.G.acc1 + gn.node[j], w2 * H[1], w2 * H[2], w2 * H[3], w2 * H[4]);
        red_add_f32(a.G.acc2 + gn.node[j], w2 * H[5]);
      }
    };
    for (int base = wfirst; base < nc; base += rstride) {
      const int p = base + grp;
      const bool valid = p < nc;
      float4 xp = make_float4(0.f, 0.f, 0.f, 0.f), q = xp, bb = xp;
      int body = 0;
      if (valid) {
        xp = a.C.xp[p];
        q = a.C.nrm[p];
        bb = a.C.bias[p];
        body = a.C.id[p].y;
      }
      GroupNodes gn;
      if (base == wfirst)
        own_nodes(gn);
      else
        group_nodes(g, xp, sub, gn);
      const float n3[3] = {q.x, q.y, q.z};
      phase_g(p, valid, xp, n3, q.w, bb, body, gn);
    }
    if (!grid_sync(B)) return;
    lap(1);

    // ---- N: step the contact nodes by alpha (v_next = v_cur + alpha dv, in
    // double-float, into the other buffer), gradient, stopping norms,
    // direction, grid line-search sums
    float2* slot = next_slot();
    {
      float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // G2, P2 - P*2, J2, A, B
      for (int t = gtid; t < ncn; t += gstride) {
        const int node = t == gtid ? my_node : a.G.cnodes[t];
        const float4 vs = a.G.vs[node];
        const float m = vs.w;
        float4 v = vcur[node];
        float4 vl = lcur[node];
        if (it > 0) {
          const float4 d = a.G.dv[node];
          dd_add(v.x, vl.x, al * d.x);
          dd_add(v.y, vl.y, al * d.y);
          dd_add(v.z, vl.z, al * d.z);
          vnxt[node] = v;
          lnxt[node] = vl;
        }
        float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
        // written by other blocks' reductions in this launch: read from L2
        const float4 c0 = __ldcg(a.G.acc0 + node);
        const float4 c1 = __ldcg(a.G.acc1 + node);
        const float c2 = __ldcg(a.G.acc2 + node);
        a.G.acc0[node] = make_float4(0.f, 0.f, 0.f, 0.f);
        a.G.acc1[node] = make_float4(0.f, 0.f, 0.f, 0.f);
        a.G.acc2[node] = 0.f;
        if (m > 0.f && v.w == 0.f) {  // free DoF (v.w flags a Dirichlet node)
          // v - v* with the low part of the iterate
          const float r0 = (v.x - vs.x) + vl.x, r1 = (v.y - vs.y) + vl.y, r2 = (v.z - vs.z) + vl.z;
          const float g0 = m * r0 + c0.x, g1 = m * r1 + c0.y, g2 = m * r2 + c0.z;
          const float inv_m = 1.0f / m;
          acc[0] += (g0 * g0 + g1 * g1 + g2 * g2) * inv_m;
          // m (|v|^2 - |v*|^2) = m r . (2 v* + r)
          acc[1] += m * (r0 * (2.f * vs.x + r0) + r1 * (2.f * vs.y + r1) + r2 * (2.f * vs.z + r2));
          acc[2] += (c0.x * c0.x + c0.y * c0.y + c0.z * c0.z) * inv_m;
          // H = m I + contact block; dv = -H^-1 g (Cholesky)
          const float h00 = m + c0.w, h11 = m + c1.x, h22 = m + c1.y;
          const float h01 = c1.z, h02 = c1.w, h12 = c2;
          const float l00 = sqrtf(h00);
          const float l10 = h01 / l00, l20 = h02 / l00;
          const float l11 = sqrtf(fmaxf(h11 - l10 * l10, 1e-30f));
          const float l21 = (h12 - l20 * l10) / l11;
          const float l22 = sqrtf(fmaxf(h22 - l20 * l20 - l21 * l21, 1e-30f));
          const float y0 = -g0 / l00;
          const float y1 = (-g1 - l10 * y0) / l11;
          const float y2 = (-g2 - l20 * y0 - l21 * y1) / l22;
          dv.z = y2 / l22;
          dv.y = (y1 - l21 * dv.z) / l11;
          dv.x = (y0 - l10 * dv.y - l20 * dv.z) / l00;
          acc[3] += m * (dv.x * dv.x + dv.y * dv.y + dv.z * dv.z);
          acc[4] += m * (dv.x * r0 + dv.y * r1 + dv.z * r2);
        }
        a.G.dv[node] = dv;
      }
      if (it > 0) {
        float4* t = vcur; vcur = vnxt; vnxt = t;
        t = lcur; lcur = lnxt; lnxt = t;
      }
      float acc6[6] = {acc[0], acc[1], acc[2], acc[3], acc[4], 0.f};
      if (!reduce_all(acc6, slot, B, s_red, s_tot, next_cpart())) return;
    }
    lap(2);
    // stopping test (Alg. 1). The scalar logic runs in thread 0 of each block
    // (FP64 is a narrow pipe on GB300) and the decision is broadcast; every
    // block computes it from the same totals, so all decide alike.
    if (tid == 0) {
      const float2 A = s_tot[3], Bs = s_tot[4];
      const float G2 = s_tot[0].x + s_tot[0].y, J2 = s_tot[2].x + s_tot[2].y;
      const float P2 = (pstar2_hi + s_tot[1].x) + (pstar2_lo + s_tot[1].y);
      const float Gn = sqrtf(G2), Pn = sqrtf(fmaxf(P2, 0.f)), Jn = sqrtf(J2);
      const float mx = fmaxf(Pn, Jn);
      resid = mx > 0.f ? Gn / mx : 0.f;
      int dec = 0;
      if (!(G2 == G2) || !(A.x == A.x) || !(Bs.x == Bs.x)) {
        if (block == 0) atomicOr(a.status, kStNan);
        dec = 1;
      } else if (Gn < eps_a + eps_r * mx || G2 == 0.f) {
        dec = 1;  // converged
      } else if (it >= a.max_iters) {
        if (block == 0) atomicOr(a.status, kStNotConverged);
        dec = 1;
      }
      s_dec = dec;
      s_A = A;
      s_B = Bs;
    }
    if (tid < 32) {
      ls.reset();
      if (tid < kLsPoints) s_pts[tid] = ls.pt;
    }
    __syncthreads();
    if (s_dec) break;

    // ---- C: dv_c = J dv (kGrp lanes per contact)
    for (int base = wfirst; base < nc; base += rstride) {
      const int p = base + grp;
      const bool valid = p < nc;
      GroupNodes gn;
      if (base == wfirst)
        own_nodes(gn);
      else
        group_nodes(g, valid ? a.C.xp[p] : make_float4(0.f, 0.f, 0.f, 0.f), sub, gn);
      float e[3] = {0.f, 0.f, 0.f};
      if (valid) {
        float4 dq[kGrpNodes];
#pragma unroll
        for (int j = 0; j < kGrpNodes; ++j)
          if (sub + kGrp * j < 27) dq[j] = __ldcg(a.G.dv + gn.node[j]);
#pragma unroll
        for (int j = 0; j < kGrpNodes; ++j) {
          if (sub + kGrp * j >= 27) continue;
          e[0] = fmaf(gn.w[j], dq[j].x, e[0]);
          e[1] = fmaf(gn.w[j], dq[j].y, e[1]);
          e[2] = fmaf(gn.w[j], dq[j].z, e[2]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 1; o < kGrp; o <<= 1) e[c] += __shfl_xor_sync(0xffffffffu, e[c], o);
      if (valid && sub == 0) a.C.dvc[p] = make_float4(e[0], e[1], e[2], 0.f);
    }
    if (!grid_sync(B)) return;
    // ---- L: line-search passes of 8 points each (thread per contact)
    for (int pass = 0;; ++pass) {
      float2* sl = local_ls ? nullptr : next_slot();
      float alphas[kLsPoints];
#pragma unroll
      for (int k = 0; k < kLsPoints; ++k) alphas[k] = s_pts[k];
      float acc[2 * kLsPoints];
#pragma unroll
      for (int k = 0; k < 2 * kLsPoints; ++k) acc[k] = 0.f;
      int k = 0;
      for (int p = ls_first; p < nc; p += ls_stride, ++k) {
        const int slot = k * kThreads + tid;
        ContactLine L;
        if (pass > 0 && k < kLsCacheDepth) {
          line_load(s_line, slot, s_body, a.h, eps2, L);
        } else {
          float4 xp; float n[3]; float n0;
          load_contact(a.C, p, xp, n, n0);
          const int b = a.C.id[p].y;
          const DevBody& bd = s_body[b];
          // written by other blocks in phases G and C: read from L2
          const float4 vc = __ldcg(a.C.vc + p), q = __ldcg(a.C.dvc + p);
          const float e[3] = {q.x, q.y, q.z};
          const float u[3] = {vc.x, vc.y, vc.z};
          contact_line(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u, e, L);
          if (k < kLsCacheDepth) line_store(s_line, slot, L, b);
        }
#pragma unroll
        for (int j = 0; j < kLsPoints; ++j) {
          float d1, d2;
          contact_line_eval(L, alphas[j], d1, d2);
          acc[j] += d1;
          acc[kLsPoints + j] += d2;
        }
      }
      if (!reduce_all(acc, sl, local_ls ? Bl : B, s_red, s_tot, local_ls ? nullptr : next_cpart()))
        return;
      ++ls_passes;
      if (tid < 32) {
        const int st = ls.update(s_tot, s_A, s_B, a.ls_rel_tol, pass + 1 >= a.ls_max_iters);
        if (tid == 0) {
          if (st == LineSearch::kFailed && block == 0) atomicOr(a.status, kStLineSearch);
          s_dec = st != LineSearch::kMore;
          s_alpha = ls.best;
        }
        if (tid < kLsPoints) s_pts[tid] = ls.pt;
      }
      __syncthreads();
      if (s_dec) break;
    }
    lap(3);
    alpha = s_alpha;
    ++it;
    if (alpha == 0.f) break;  // no further progress possible at this precision
  }
  // no block of a cluster leaves while another may still read its shared memory
  if (kCluster) cluster_sync_all();

  // the solution must end in G.v, which G2P reads; release the node flags
  for (int t = gtid; t < ncn; t += gstride) {
    const int node = t == gtid ? my_node : a.G.cnodes[t];
    if (vcur != a.G.v) a.G.v[node] = vcur[node];
    a.G.cflag[node] = 0;
  }
  // ---- impulses at the solution: gamma = -dl_c/dv_c on the particle; the
  // body receives -gamma and its moment about the body origin (Eq. (3));
  // each warp sums its contacts body by body before the block's shared sums
  for (int p0 = gtid & ~31; p0 < nc; p0 += gstride) {
    const int p = p0 + lane;
    int b = -1;
    float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (p < nc) {
      float4 xp; float n[3]; float n0;
      load_contact(a.C, p, xp, n, n0);
      b = a.C.id[p].y;
      const DevBody& bd = s_body[b];
      const float4 vc = __ldcg(a.C.vc + p);
      const float u[3] = {vc.x, vc.y, vc.z};
      ContactLaw L;
      contact_law(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u, L);
      float gr[3];
      contact_grad(L, n, gr);
      a.C.gamma[p] = make_float4(-gr[0], -gr[1], -gr[2], 0.f);
      const float r0 = xp.x - bd.p[0], r1 = xp.y - bd.p[1], r2 = xp.z - bd.p[2];
      q[0] = gr[0]; q[1] = gr[1]; q[2] = gr[2];
      q[3] = r1 * gr[2] - r2 * gr[1];
      q[4] = r2 * gr[0] - r0 * gr[2];
      q[5] = r0 * gr[1] - r1 * gr[0];
    }
    unsigned left = __ballot_sync(0xffffffffu, b >= 0);
    while (left) {  // one body of the warp at a time (mostly a single one)
      const int bb = __shfl_sync(0xffffffffu, b, __ffs(left) - 1);
      const bool mine = b == bb;
      float t[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        t[c] = mine ? q[c] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t[c] += __shfl_xor_sync(0xffffffffu, t[c], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) atomicAdd(&s_imp[bb][c], t[c]);
      }
      left &= ~__ballot_sync(0xffffffffu, mine);
    }
  }
  __syncthreads();
  for (int i = tid; i < a.nb * 6; i += kThreads) {
    const float v = (&s_imp[0][0])[i];
    if (v != 0.f) atomicAdd(a.impulses + i, (double)v);
  }
  lap(4);
  if (gtid == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) atomicAdd(&a.stats->solve_ns[k], tph[k]);
    atomicAdd(&a.stats->iters_total, it);
    atomicMax(&a.stats->iters_max, it);
    atomicAdd(&a.stats->ls_evals_total, ls_passes);
    if (!local_ls) atomicAdd(&a.stats->ls_split, 1);
    if (kCluster) atomicAdd(&a.stats->cluster, 1);
    atomicMax(&a.stats->cnodes_max, ncn);
    atomicMax(reinterpret_cast<int*>(&a.stats->residual_max), __float_as_int(resid));
  }
}

template <bool kCluster>
__global__ void __launch_bounds__(kThreads, 1) k_solve(SolveArgs a) {
  solve_body<kCluster>(a, (int)blockIdx.x, (int)gridDim.x);
}

// Batched: scene order[b / kBlocks] is solved by blocks b of one cluster of
// kBlocks (one block: its reductions need no barrier beyond __syncthreads;
// more: a thread-block cluster per scene, as the single-scene cluster solve).
// `order` lists the scenes largest first, so that the long solves start in the
// first wave of blocks.
template <int kBlocks>
__global__ void __launch_bounds__(kThreads, 1) k_solve_batch(const SolveArgs* __restrict__ args,
                                                             const int* __restrict__ order) {
  __shared__ SolveArgs s_a;
  load_args(args + order[blockIdx.x / kBlocks], s_a);
  __syncthreads();
  if (threadIdx.x == 0) s_a.cluster_max = kBlocks > 1 ? 0x7fffffff : 0;  // this launch's kind
  __syncthreads();
  if constexpr (kBlocks == 1)
    solve_body<false>(s_a, 0, 1);
  else
    solve_body<true>(s_a, (int)(blockIdx.x % kBlocks), kBlocks);
}

// ---------------------------------------------------------------------------
// Adjoint of the contact solve: implicit differentiation of the optimality
// condition of Eq. (8)-(9) at the last substep's solution v,
//   grad l_p = M (v - v*) + J^T dl_c(J v + b) = 0   (free DoFs).
// For a loss L(v) with vbar = dL/dv, lambda solves H^ lambda = vbar on the
// free DoFs, with H^ = M + J^T (d2 l_c) J the exact Hessian (the blocks of
// Eq. (10) plus their couplings between nodes), and
//   dL/dv*    = M lambda on free DoFs; vbar - (J^T d2l_c J lambda) on the
//               other nodes (Dirichlet or massless: v = v* there),
//   dL/dv_r   = d2l_c (J lambda)_c   (the contact velocity has b = -v_r(x_p)),
//   dL/dmu_c  = -(n0 / s) u_t . (J lambda)_c   (d/dmu of dl_c, Sec. IV-B).
// H^ is symmetric positive definite (M > 0 on free DoFs, d2 l_c positive
// semidefinite), so lambda comes from conjugate gradients preconditioned by
// the 3x3 diagonal blocks of H^, the matrix the quasi-Newton iteration
// inverts (Eq. (10)). Only contact nodes take part: elsewhere H^ = M, so
// lambda = M^-1 vbar and dL/dv* = vbar.
//
// Per CG iteration (one cooperative launch, like the forward solve):
//   A  contacts: y_c = d2l_c J (z + beta p), scattered as w y_c;
//   B  contact nodes: p = z + beta p, q = M p + J^T y; sum p.q;
//   C  contact nodes: x += a p, r -= a q, z = P^-1 r; sum r.z.
// CG runs in FP32 inside a mixed-precision iterative refinement: lambda is
// kept as a double-float pair and the residual vbar - H^ lambda that starts
// each round (and decides convergence) is formed in FP64.
// The contact-node list is rebuilt here (the forward solve releases its
// own); its node flags hold list positions + 1 for the duration of the call.

// per-node vectors of the adjoint, each cnodes_cap float4 apart
// (kVD and the slot after it hold 4 doubles per node)
enum { kVRhs = 0, kVX, kVR, kVZ, kVP, kVQ, kVAcc, kVL0, kVL1, kVXh, kVXl, kVD, kVD2, kAdjVectors };
constexpr int kRefineRounds = 3;  // FP32 CG rounds of the iterative refinement
static_assert(kAdjVectors == kAdjointVectors, "adjoint vector count");

// The contact Hessian at the stored solution velocity, kept in factored form
// d2l_c = N'' n n^T + (mu n0 / s) (I - n n^T - u_t u_t^T / s^2) and applied
// as such: the stiff normal term then never rounds into the tangential
// components, which stay accurate to the (much smaller) friction scale.
struct AdjHess {
  float n[3], ut[3];
  float dN, d2N, cs, inv_s2;
  float n0;
  float n0_s;  // n0 / s, for dL/dmu
};

__device__ __forceinline__ void adjoint_contact(const Contacts& C, int p, const DevBody* bodies,
                                                float h, float eps_s, AdjHess& A, int& body,
                                                float4& xp) {
  float n0;
  load_contact(C, p, xp, A.n, n0);
  body = C.id[p].y;
  const DevBody& bd = bodies[body];
  const float4 vc = C.vc[p];
  const float u[3] = {vc.x, vc.y, vc.z};
  ContactLaw L;
  contact_law(xp.w, n0, bd.mu, bd.k, bd.d, h, eps_s, A.n, u, L);
  // u_t = u - (u.n) n keeps a normal component of the order of ulp(|u|)
  // from rounding; near sticking, where |u_t| ~ eps_s << |u|, that component
  // would mix the large normal part of J lambda into the friction terms, so
  // project it out once more
  const float tn = L.ut[0] * A.n[0] + L.ut[1] * A.n[1] + L.ut[2] * A.n[2];
#pragma unroll
  for (int r = 0; r < 3; ++r) A.ut[r] = L.ut[r] - tn * A.n[r];
  A.dN = L.dN;
  A.d2N = L.d2N;
  A.cs = L.cs;
  A.inv_s2 = L.inv_s2;
  A.n0 = n0;
  A.n0_s = n0 * sqrtf(L.inv_s2);
}

// Gradient of w_ip (physical units) at the lane's stencil node (lane_node's
// node order; zero for lanes >= 27).
__device__ __forceinline__ void lane_weight_grad(const GridDev& g, const float4& xp, int lane,
                                                 float (&gw)[3]) {
  Stencil s;
  stencil(g, xp.x, xp.y, xp.z, s);
  const int l = lane < 27 ? lane : 0;
  const int c[3] = {l % 3, (l / 3) % 3, l / 9};
  float dw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float f = s.fx[a];
    dw[a] = (c[a] == 0 ? -(1.5f - f) : c[a] == 1 ? -2.0f * (f - 1.0f) : (f - 0.5f)) * g.inv_dx;
  }
  const float w0 = s.w[0][c[0]], w1 = s.w[1][c[1]], w2 = s.w[2][c[2]];
  const float on = lane < 27 ? 1.0f : 0.0f;
  gw[0] = on * dw[0] * w1 * w2;
  gw[1] = on * w0 * dw[1] * w2;
  gw[2] = on * w0 * w1 * dw[2];
}

// Adjoint of the contact's inputs to the solve, given xi = J lambda and
// y = d2l_c xi (FP64). With theta_bar = -(d grad l_c / d theta)^T xi
// (implicit differentiation of Eq. (9)) for the lagged depth phi0, the lagged
// normal impulse n0, the normal n and the bias b = -v_r(x_p) of Sec. IV-B,
// V-B, and their dependence on the particle's start-of-substep position and
// velocity (phi0 = -sdf(x_p), n = grad sdf(x_p), n0 = gamma_n(phi0, n.(v_p -
// v_r(x_p))), v_r(x) = v + omega x (x - p)): the adjoint of x_p (without the
// stencil-weight term) and of v_p.
__device__ void contact_input_adjoint(const AdjHess& A, const DevBody& bd, const float4& xp,
                                      const float4& vc, const float4& bias, const float (&vp)[3],
                                      float h, const double (&xi)[3], const double (&y)[3],
                                      float (&xb)[3], float (&vb)[3], double (&rot)[3],
                                      double (&wdir)[3]) {
  const double n[3] = {A.n[0], A.n[1], A.n[2]}, t[3] = {A.ut[0], A.ut[1], A.ut[2]};
  const double u[3] = {vc.x, vc.y, vc.z};
  const double un = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
  const double nxi = n[0] * xi[0] + n[1] * xi[1] + n[2] * xi[2];
  const double txi = t[0] * xi[0] + t[1] * xi[1] + t[2] * xi[2];
  const double hk = (double)h * (double)bd.k, d = bd.d;
  const double cs = A.cs, inv_s2 = A.inv_s2, inv_s = sqrt(inv_s2);
  const double bbar[3] = {-y[0], -y[1], -y[2]};
  const double n0bar = -(double)bd.mu * inv_s * txi;
  // the normal law is active where N' < 0 (v_n below its cutoff)
  double phi0bar = A.dN < 0.f ? hk * (1.0 - d * un) * nxi : 0.0;
  double nbar[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    nbar[r] = -((double)A.d2N * nxi * u[r] + (double)A.dN * xi[r] + cs * un * txi * inv_s2 * t[r] -
                cs * nxi * u[r] - cs * un * xi[r]);
  // lagged normal impulse n0 = h k (phi0 - h vn0) (1 - d vn0), vn0 = n . (v_p - v_r)
  const double rel[3] = {(double)vp[0] + bias.x, (double)vp[1] + bias.y, (double)vp[2] + bias.z};
  const double vn0 = n[0] * rel[0] + n[1] * rel[1] + n[2] * rel[2];
  const double a0 = (double)xp.w - h * vn0, c0 = 1.0 - d * vn0;
  double vn0bar = 0.0;
  if (a0 > 0.0 && c0 > 0.0) {
    phi0bar += n0bar * hk * c0;
    vn0bar = n0bar * hk * (-(double)h * c0 - d * a0);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    vb[r] = (float)(vn0bar * n[r]);
    nbar[r] += vn0bar * rel[r];
  }
  const double w[3] = {bd.w[0], bd.w[1], bd.w[2]};
  const double wxb[3] = {w[1] * bbar[2] - w[2] * bbar[1], w[2] * bbar[0] - w[0] * bbar[2],
                         w[0] * bbar[1] - w[1] * bbar[0]};
  const double wxn[3] = {w[1] * n[2] - w[2] * n[1], w[2] * n[0] - w[0] * n[2], w[0] * n[1] - w[1] * n[0]};
  // (d n / d x)^T nbar: sphere (I - n n^T) / dist, capsule side (I - n n^T - a a^T) / dist
  double dn[3] = {0.0, 0.0, 0.0};
  if (bd.shape == MPM_SPHERE || bd.shape == MPM_CAPSULE) {
    const double r[3] = {(double)xp.x - bd.p[0], (double)xp.y - bd.p[1], (double)xp.z - bd.p[2]};
    double o[3] = {r[0], r[1], r[2]};
    double ax[3] = {0.0, 0.0, 0.0};
    if (bd.shape == MPM_CAPSULE) {
      ax[0] = bd.R[2]; ax[1] = bd.R[5]; ax[2] = bd.R[8];
      const double z = ax[0] * r[0] + ax[1] * r[1] + ax[2] * r[2];
      const double L = bd.prm[0];
      const double cz = z < -L ? -L : (z > L ? L : z);
#pragma unroll
      for (int c = 0; c < 3; ++c) o[c] = r[c] - cz * ax[c];
      if (!(z > -L && z < L)) ax[0] = ax[1] = ax[2] = 0.0;  // a cap: sphere-like
    }
    const double dist = sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
    if (dist > 0.0) {
      const double nn = n[0] * nbar[0] + n[1] * nbar[1] + n[2] * nbar[2];
      const double an = ax[0] * nbar[0] + ax[1] * nbar[1] + ax[2] * nbar[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) dn[c] = (nbar[c] - nn * n[c] - an * ax[c]) / dist;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
    xb[c] = (float)(-phi0bar * n[c] + wxb[c] + vn0bar * wxn[c] + dn[c]);
  // The body's orientation (a rotation dtheta about p): the body-frame point
  // moves as x would by r x dtheta (r = x_p - p), which the depth and the
  // normal's x-dependence see, and the normal turns with the body
  // (dn = dtheta x n); the bias does not depend on it. Left-perturbation
  // adjoint: rot = (-phi0bar n + dn) x r + n x nbar.
  const double r[3] = {(double)xp.x - bd.p[0], (double)xp.y - bd.p[1], (double)xp.z - bd.p[2]};
  const double g[3] = {-phi0bar * n[0] + dn[0], -phi0bar * n[1] + dn[1], -phi0bar * n[2] + dn[2]};
  rot[0] = g[1] * r[2] - g[2] * r[1] + n[1] * nbar[2] - n[2] * nbar[1];
  rot[1] = g[2] * r[0] - g[0] * r[2] + n[2] * nbar[0] - n[0] * nbar[2];
  rot[2] = g[0] * r[1] - g[1] * r[0] + n[0] * nbar[1] - n[1] * nbar[0];
  // the angular velocity through the lagged normal impulse:
  // vn0 = n . (v_p - v - omega x r) -> -vn0bar (r x n)
  wdir[0] = -vn0bar * (r[1] * n[2] - r[2] * n[1]);
  wdir[1] = -vn0bar * (r[2] * n[0] - r[0] * n[2]);
  wdir[2] = -vn0bar * (r[0] * n[1] - r[1] * n[0]);
}

// The cotangent of the contact's gradient dl_c (the impulse the body
// receives, minus the particle's) from the body's impulse and moment
// cotangents: ghat = Jbar + Lbar x r, r = x_p - p (Eq. (3)).
__device__ __forceinline__ void impulse_cotangent(const double* bg, const DevBody& bd,
                                                  const float4& xp, double (&gh)[3]) {
  const double r[3] = {(double)xp.x - bd.p[0], (double)xp.y - bd.p[1], (double)xp.z - bd.p[2]};
  gh[0] = bg[0] + bg[4] * r[2] - bg[5] * r[1];
  gh[1] = bg[1] + bg[5] * r[0] - bg[3] * r[2];
  gh[2] = bg[2] + bg[3] * r[1] - bg[4] * r[0];
}

// y = d2l_c u (FP32)
__device__ __forceinline__ void hess_apply(const AdjHess& A, const float (&u)[3], float (&y)[3]) {
  const float un = A.n[0] * u[0] + A.n[1] * u[1] + A.n[2] * u[2];
  const float tu = (A.ut[0] * u[0] + A.ut[1] * u[1] + A.ut[2] * u[2]) * A.inv_s2;
#pragma unroll
  for (int r = 0; r < 3; ++r) y[r] = A.d2N * un * A.n[r] + A.cs * ((u[r] - un * A.n[r]) - tu * A.ut[r]);
}

// y = d2l_c u (FP64, same factors)
__device__ __forceinline__ void hess_apply(const AdjHess& A, const double (&u)[3], double (&y)[3]) {
  const double n[3] = {A.n[0], A.n[1], A.n[2]}, t[3] = {A.ut[0], A.ut[1], A.ut[2]};
  const double un = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
  const double tu = (t[0] * u[0] + t[1] * u[1] + t[2] * u[2]) * (double)A.inv_s2;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    y[r] = (double)A.d2N * un * n[r] + (double)A.cs * ((u[r] - un * n[r]) - tu * t[r]);
}

// the 3x3 block (xx yy zz xy xz yz), for the preconditioner
__device__ __forceinline__ void hess_block(const AdjHess& A, float (&H)[6]) {
  auto e = [&](int r, int c) {
    const float id = (r == c) ? 1.0f : 0.0f;
    return A.d2N * A.n[r] * A.n[c] + A.cs * (id - A.n[r] * A.n[c] - A.ut[r] * A.ut[c] * A.inv_s2);
  };
  H[0] = e(0, 0); H[1] = e(1, 1); H[2] = e(2, 2);
  H[3] = e(0, 1); H[4] = e(0, 2); H[5] = e(1, 2);
}

// z = P^-1 r with P = L L^T stored as (l10, l20, l21, 1/l00), (1/l11, 1/l22, free, m)
__device__ __forceinline__ float4 chol_apply(const float4 a, const float4 b, const float4 r) {
  const float y0 = r.x * a.w;
  const float y1 = (r.y - a.x * y0) * b.x;
  const float y2 = (r.z - a.y * y0 - a.z * y1) * b.y;
  const float z2 = y2 * b.y;
  const float z1 = (y1 - a.z * z2) * b.x;
  const float z0 = (y0 - a.x * z1 - a.y * z2) * a.w;
  return make_float4(z0, z1, z2, 0.f);
}

__device__ __forceinline__ double warp_sum_f64(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// lambda = hi + lo at list position ci (zero off the list)
__device__ __forceinline__ void lambda_at(const float4* xh, const float4* xl, int ci, double (&x)[3]) {
  x[0] = x[1] = x[2] = 0.0;
  if (ci >= 0) {
    const float4 h = __ldcg(xh + ci), l = __ldcg(xl + ci);
    x[0] = (double)h.x + (double)l.x;
    x[1] = (double)h.y + (double)l.y;
    x[2] = (double)h.z + (double)l.z;
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_adjoint(AdjointArgs a) {
  __shared__ DevBody s_body[kMaxBodies];
  __shared__ float s_red[kWarps][kRedWidth];
  __shared__ float2 s_tot[kRedWidth];
  __shared__ double s_bb[kMaxBodies][kAdjBodySlots];  // FP64: the per-body sums cancel strongly
  const int tid = threadIdx.x;
  // the last substep's contact count (G2P has reset the live counter), or
  // in mpm_backward mode the live count of the substep just solved
  const int count = a.gbar ? *a.C.count : a.stats->last_contacts;
  const int nc = count < a.C.cap ? count : a.C.cap;
  int nblk = (nc + kAdjContactsPerBlock - 1) / kAdjContactsPerBlock;
  nblk = nblk < (int)gridDim.x ? nblk : (int)gridDim.x;
  nblk = nblk < kMaxSolveBlocks ? nblk : kMaxSolveBlocks;
  nblk = nblk > 1 ? nblk : 1;
  if ((int)blockIdx.x >= nblk) return;
  for (int i = tid; i < a.nb * (int)(sizeof(DevBody) / 4); i += kThreads)
    reinterpret_cast<float*>(s_body)[i] = reinterpret_cast<const float*>(a.bodies)[i];
  for (int i = tid; i < kMaxBodies * kAdjBodySlots; i += kThreads) (&s_bb[0][0])[i] = 0.0;
  __syncthreads();
  Barrier B{a.bar, (unsigned)nblk, a.status, a.poison, 0, 0u, (unsigned)blockIdx.x};
  const int gtid = blockIdx.x * kThreads + tid;
  const int gstride = nblk * kThreads;
  const int lane = tid & 31;
  const int gwarp = gtid >> 5;
  const int nwarps = gstride >> 5;
  const GridDev& g = a.g;
  const size_t cap = (size_t)a.G.cnodes_cap;
  float4* vRhs = a.vec + kVRhs * cap;
  float4* vX = a.vec + kVX * cap;
  float4* vR = a.vec + kVR * cap;
  float4* vZ = a.vec + kVZ * cap;
  float4* vP = a.vec + kVP * cap;
  float4* vQ = a.vec + kVQ * cap;
  float4* vAcc = a.vec + kVAcc * cap;
  float4* vL0 = a.vec + kVL0 * cap;
  float4* vL1 = a.vec + kVL1 * cap;
  float4* vXh = a.vec + kVXh * cap;
  float4* vXl = a.vec + kVXl * cap;
  double* acc64 = reinterpret_cast<double*>(a.vec + kVD * cap);  // 4 doubles per node
  int rslot = 0;
  auto next_slot = [&]() -> float2* {
    float2* s = reinterpret_cast<float2*>(a.red) + (size_t)(rslot & 3) * kMaxSolveBlocks * kRedWidth;
    ++rslot;
    return s;
  };
  const int n_nodes_total = g.rx * g.ry * g.rz;
  auto node_of_id = [&](int id) -> int {
    if (id < 0 || id >= n_nodes_total) return -1;
    const int i = id % g.rx, j = (id / g.rx) % g.ry, k = id / (g.rx * g.ry);
    const int node = node_index(g, i, j, k);  // negative: a sparse grid's unmapped block
    return node < 0 ? -1 : node;
  };
  auto list_pos = [&](const LaneNode& ln) -> int {
    return lane < 27 ? __ldcg(a.G.cflag + ln.node) - 1 : -1;
  };

  // a solve that gave up at a barrier left node flags and accumulators behind
  if (__ldcg(a.poison)) {
    const size_t n_nodes = (size_t)storage_nodes(g);
    for (size_t t = gtid; t < n_nodes; t += gstride) {
      a.G.cflag[t] = 0;
      a.G.acc0[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.G.acc1[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.G.acc2[t] = 0.f;
    }
    if (!grid_sync(B)) return;
    if (gtid == 0) *a.poison = 0;
  }

  // ---- contact-node list; flags hold list position + 1 (-1: claimed, no room)
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int p = gtid; p < nc; p += gstride) {
    const float4 xp = a.C.xp[p];
    Stencil s;
    stencil(g, xp.x, xp.y, xp.z, s);
    int node[27];
    unsigned won = 0u;
#pragma unroll
    for (int c = 0; c < 27; ++c) {
      node[c] = node_index(g, s.base[0] + c % 3, s.base[1] + (c / 3) % 3, s.base[2] + c / 9);
      if (atomicCAS(a.G.cflag + node[c], 0, -1) == 0) won |= 1u << c;
    }
    if (won) {
      int slot = atomicAdd(a.G.n_cnodes, __popc(won));
#pragma unroll
      for (int c = 0; c < 27; ++c)
        if ((won >> c) & 1u) {
          if (slot < a.G.cnodes_cap) {
            a.G.cnodes[slot] = node[c];
            a.G.cflag[node[c]] = slot + 1;
            if (a.gbar) {
              const float4 gb = a.gbar[node[c]];
              vRhs[slot] = make_float4(gb.x, gb.y, gb.z, 0.f);
            } else {
              vRhs[slot] = zero4;
            }
            vL0[slot] = zero4;
            vL1[slot] = zero4;
            vAcc[slot] = zero4;
            double* d = acc64 + 4 * (size_t)slot;
            d[0] = d[1] = d[2] = d[3] = 0.0;
          } else {  // unreachable (the list holds every grid node): flag and clean up
            atomicOr(a.status, kStCapacity);
            atomicExch(a.poison, 1);
          }
          ++slot;
        }
    }
  }
  if (!grid_sync(B)) return;
  int ncn = __ldcg(a.G.n_cnodes);
  ncn = ncn < a.G.cnodes_cap ? ncn : a.G.cnodes_cap;

  // ---- vbar onto the contact nodes; diagonal blocks of J^T d2l_c J (w^2 H)
  for (int i = gtid; i < a.n_in; i += gstride) {
    const int node = node_of_id(a.ids[i]);
    if (node < 0) {
      atomicOr(a.status, 1u << MPM_ERR_INVALID_ARG);
      continue;
    }
    const int ci = __ldcg(a.G.cflag + node) - 1;
    if (ci >= 0) {
      float* d = reinterpret_cast<float*>(vRhs + ci);
      atomicAdd(d, a.vbar[3 * i]);
      atomicAdd(d + 1, a.vbar[3 * i + 1]);
      atomicAdd(d + 2, a.vbar[3 * i + 2]);
    }
  }
  for (int p = gwarp; p < nc; p += nwarps) {
    AdjHess A;
    int body;
    float4 xp;
    adjoint_contact(a.C, p, s_body, a.h, a.eps_s, A, body, xp);
    const LaneNode ln = lane_node(g, xp, lane);
    const int ci = list_pos(ln);
    if (ci >= 0) {
      float H[6];
      hess_block(A, H);
      const float w2 = ln.w * ln.w;
      red_add_v4(vL0 + ci, w2 * H[0], w2 * H[1], w2 * H[2], w2 * H[3]);
      red_add_v4(vL1 + ci, w2 * H[4], w2 * H[5], 0.f, 0.f);
      if (a.body_gbar) {
        // the body's impulse depends on the solution through dl_c(J v + b):
        // vbar += J^T d2l_c ghat
        double gh[3], y[3];
        impulse_cotangent(a.body_gbar + 6 * body, s_body[body], xp, gh);
        hess_apply(A, gh, y);
        float* d = reinterpret_cast<float*>(vRhs + ci);
        atomicAdd(d, (float)(ln.w * y[0]));
        atomicAdd(d + 1, (float)(ln.w * y[1]));
        atomicAdd(d + 2, (float)(ln.w * y[2]));
      }
    }
  }
  if (!grid_sync(B)) return;

  // ---- preconditioner P = m I + block (Cholesky), r = vbar (free DoFs),
  // lambda = 0, increment x = 0
  {
    float acc[1] = {0.f};  // r.z
    for (int t = gtid; t < ncn; t += gstride) {
      const int node = a.G.cnodes[t];
      const float m = a.G.vs[node].w;
      const bool fre = m > 0.f && a.G.v[node].w == 0.f;
      const float4 c0 = __ldcg(vL0 + t), c1 = __ldcg(vL1 + t);
      float4 L0 = zero4, L1 = make_float4(0.f, 0.f, 0.f, m);
      float4 r = zero4, z = zero4;
      if (fre) {
        const float h00 = m + c0.x, h11 = m + c0.y, h22 = m + c0.z;
        const float h01 = c0.w, h02 = c1.x, h12 = c1.y;
        const float l00 = sqrtf(h00);
        const float l10 = h01 / l00, l20 = h02 / l00;
        const float l11 = sqrtf(fmaxf(h11 - l10 * l10, 1e-30f));
        const float l21 = (h12 - l20 * l10) / l11;
        const float l22 = sqrtf(fmaxf(h22 - l20 * l20 - l21 * l21, 1e-30f));
        L0 = make_float4(l10, l20, l21, 1.0f / l00);
        L1 = make_float4(1.0f / l11, 1.0f / l22, 1.f, m);
        r = __ldcg(vRhs + t);
        r.w = 0.f;
        z = chol_apply(L0, L1, r);
        acc[0] += r.x * z.x + r.y * z.y + r.z * z.z;
      }
      vL0[t] = L0;
      vL1[t] = L1;
      vR[t] = r;
      vZ[t] = z;
      vX[t] = zero4;
      vP[t] = zero4;
      vXh[t] = zero4;
      vXl[t] = zero4;
    }
    if (!reduce_all(acc, next_slot(), B, s_red, s_tot)) return;
  }
  const float rz_ref = s_tot[0].x + s_tot[0].y;  // |vbar|^2 in the P^-1 norm
  const float tol2 = (float)(a.eps_r * a.eps_r) * rz_ref;
  float rz = rz_ref;
  float rz_true = rz_ref;
  int it = 0;
  // the warp's first contact, kept in registers across the iterations
  const bool own = gwarp < nc;
  AdjHess own_A{};
  LaneNode own_ln{0, 0.f};
  int own_ci = -1;
  if (own) {
    int body;
    float4 xp;
    adjoint_contact(a.C, gwarp, s_body, a.h, a.eps_s, own_A, body, xp);
    own_ln = lane_node(g, xp, lane);
    own_ci = list_pos(own_ln);
  }

  // J^T d2l_c J lambda in FP64 onto acc64 (lambda = hi + lo)
  auto hessian_lambda_f64 = [&](const AdjHess& A, const LaneNode& ln, int ci, double (&u)[3],
                                double (&y)[3]) {
    double x[3];
    lambda_at(vXh, vXl, ci, x);
    const double w = (double)ln.w;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = warp_sum_f64(w * x[c]);
    hess_apply(A, u, y);
    if (ci >= 0) {
      double* d = acc64 + 4 * (size_t)ci;
      atomicAdd(d, w * y[0]);
      atomicAdd(d + 1, w * y[1]);
      atomicAdd(d + 2, w * y[2]);
    }
  };

  // Mixed-precision iterative refinement: each round runs FP32 conjugate
  // gradients on H^ x = r from x = 0, adds x to lambda (double-float), and
  // forms the true residual r = vbar - H^ lambda in FP64 for the next round.
  // FP32 CG alone stalls where the stiff normal blocks dominate H^ (its
  // attainable accuracy is ~1e-7 of |H^| |lambda|, and the tangential parts
  // of J lambda that dL/dmu reads are much smaller than the normal ones).
  for (int round = 0;; ++round) {
    float beta = 0.f;
    while (rz > tol2 && rz > 0.f && it < a.max_iters) {
      // ---- A: y_c = d2l_c J (z + beta p), scattered with weights w
      auto phase_a = [&](const AdjHess& A, const LaneNode& ln, int ci) {
        float pv[3] = {0.f, 0.f, 0.f};
        if (ci >= 0) {
          const float4 z = __ldcg(vZ + ci), pp = __ldcg(vP + ci);
          pv[0] = fmaf(beta, pp.x, z.x);
          pv[1] = fmaf(beta, pp.y, z.y);
          pv[2] = fmaf(beta, pp.z, z.z);
        }
        const float u[3] = {warp_sum(ln.w * pv[0]), warp_sum(ln.w * pv[1]), warp_sum(ln.w * pv[2])};
        float y[3];
        hess_apply(A, u, y);
        if (ci >= 0) red_add_v4(vAcc + ci, ln.w * y[0], ln.w * y[1], ln.w * y[2], 0.f);
      };
      if (own) phase_a(own_A, own_ln, own_ci);
      for (int p = gwarp + nwarps; p < nc; p += nwarps) {
        AdjHess A;
        int body;
        float4 xp;
        adjoint_contact(a.C, p, s_body, a.h, a.eps_s, A, body, xp);
        const LaneNode ln = lane_node(g, xp, lane);
        phase_a(A, ln, list_pos(ln));
      }
      if (!grid_sync(B)) return;
      // ---- B: p = z + beta p, q = M p + J^T y
      {
        float acc[1] = {0.f};
        for (int t = gtid; t < ncn; t += gstride) {
          const float4 L1 = vL1[t];
          const float4 y = __ldcg(vAcc + t);
          vAcc[t] = zero4;
          float4 q = zero4, pp = zero4;
          if (L1.z != 0.f) {
            const float4 z = vZ[t], po = vP[t];
            pp = make_float4(fmaf(beta, po.x, z.x), fmaf(beta, po.y, z.y), fmaf(beta, po.z, z.z), 0.f);
            q = make_float4(fmaf(L1.w, pp.x, y.x), fmaf(L1.w, pp.y, y.y), fmaf(L1.w, pp.z, y.z), 0.f);
            acc[0] += pp.x * q.x + pp.y * q.y + pp.z * q.z;
          }
          vP[t] = pp;
          vQ[t] = q;
        }
        if (!reduce_all(acc, next_slot(), B, s_red, s_tot)) return;
      }
      const float pq = s_tot[0].x + s_tot[0].y;
      if (!(pq > 0.f)) {  // H^ is positive definite on the free DoFs: only rounding gets here
        if (blockIdx.x == 0 && tid == 0 && !(pq == pq)) atomicOr(a.status, kStNan);
        break;
      }
      const float alpha = rz / pq;
      // ---- C: x += alpha p, r -= alpha q, z = P^-1 r
      {
        float acc[1] = {0.f};
        for (int t = gtid; t < ncn; t += gstride) {
          const float4 L1 = vL1[t];
          if (L1.z == 0.f) continue;
          const float4 pp = vP[t], q = vQ[t];
          float4 x = vX[t], r = vR[t];
          x.x = fmaf(alpha, pp.x, x.x); x.y = fmaf(alpha, pp.y, x.y); x.z = fmaf(alpha, pp.z, x.z);
          r.x = fmaf(-alpha, q.x, r.x); r.y = fmaf(-alpha, q.y, r.y); r.z = fmaf(-alpha, q.z, r.z);
          const float4 z = chol_apply(vL0[t], L1, r);
          vX[t] = x;
          vR[t] = r;
          vZ[t] = z;
          acc[0] += r.x * z.x + r.y * z.y + r.z * z.z;
        }
        if (!reduce_all(acc, next_slot(), B, s_red, s_tot)) return;
      }
      const float rz_new = s_tot[0].x + s_tot[0].y;
      beta = rz > 0.f ? rz_new / rz : 0.f;
      rz = rz_new;
      ++it;
    }
    // ---- lambda += x (double-float); the next round starts from x = 0
    for (int t = gtid; t < ncn; t += gstride) {
      if (vL1[t].z == 0.f) continue;
      const float4 x = vX[t];
      float4 h = vXh[t], l = vXl[t];
      dd_add(h.x, l.x, x.x);
      dd_add(h.y, l.y, x.y);
      dd_add(h.z, l.z, x.z);
      vXh[t] = h;
      vXl[t] = l;
      vX[t] = zero4;
      vP[t] = zero4;
    }
    if (!grid_sync(B)) return;
    // ---- true residual r = vbar - M lambda - J^T d2l_c J lambda (FP64)
    if (own) {
      double u[3], y[3];
      hessian_lambda_f64(own_A, own_ln, own_ci, u, y);
    }
    for (int p = gwarp + nwarps; p < nc; p += nwarps) {
      AdjHess A;
      int body;
      float4 xp;
      adjoint_contact(a.C, p, s_body, a.h, a.eps_s, A, body, xp);
      const LaneNode ln = lane_node(g, xp, lane);
      double u[3], y[3];
      hessian_lambda_f64(A, ln, list_pos(ln), u, y);
    }
    if (!grid_sync(B)) return;
    {
      float acc[1] = {0.f};
      for (int t = gtid; t < ncn; t += gstride) {
        const float4 L1 = vL1[t];
        double* d = acc64 + 4 * (size_t)t;
        const double y[3] = {__ldcg(d), __ldcg(d + 1), __ldcg(d + 2)};
        d[0] = d[1] = d[2] = 0.0;
        if (L1.z == 0.f) continue;
        const float4 b = vRhs[t], h = vXh[t], l = vXl[t];
        const double m = (double)L1.w;
        float4 r;
        r.x = (float)((double)b.x - m * ((double)h.x + (double)l.x) - y[0]);
        r.y = (float)((double)b.y - m * ((double)h.y + (double)l.y) - y[1]);
        r.z = (float)((double)b.z - m * ((double)h.z + (double)l.z) - y[2]);
        r.w = 0.f;
        const float4 z = chol_apply(vL0[t], L1, r);
        vR[t] = r;
        vZ[t] = z;
        acc[0] += r.x * z.x + r.y * z.y + r.z * z.z;
      }
      if (!reduce_all(acc, next_slot(), B, s_red, s_tot)) return;
    }
    rz_true = s_tot[0].x + s_tot[0].y;
    rz = rz_true;
    if (!(rz_true == rz_true)) {
      if (blockIdx.x == 0 && tid == 0) atomicOr(a.status, kStNan);
      break;
    }
    if (rz_true <= tol2 || round + 1 >= kRefineRounds || it >= a.max_iters) break;
  }
  if (rz_true > tol2 && blockIdx.x == 0 && tid == 0) atomicOr(a.status, kStNotConverged);

  // ---- outputs per contact: dL/dv_r(x_p) = d2l_c J lambda, dL/dmu_c (FP64
  // from lambda = hi + lo); J^T d2l_c J lambda onto the nodes for the
  // Dirichlet / massless correction
  for (int p = gwarp; p < nc; p += nwarps) {
    AdjHess A;
    int body;
    float4 xp;
    adjoint_contact(a.C, p, s_body, a.h, a.eps_s, A, body, xp);
    const LaneNode ln = lane_node(g, xp, lane);
    const int ci = list_pos(ln);
    double u[3], yd[3];
    hessian_lambda_f64(A, ln, ci, u, yd);
    // with a body impulse cotangent ghat the contact's inputs see
    // xi - ghat in place of xi = J lambda (their adjoint is
    // -(d dl_c / d theta)^T (xi - ghat), the bias's -d2l_c (xi - ghat))
    double gh[3] = {0.0, 0.0, 0.0};
    if (a.body_gbar) {
      impulse_cotangent(a.body_gbar + 6 * body, s_body[body], xp, gh);
#pragma unroll
      for (int r = 0; r < 3; ++r) u[r] -= gh[r];
      hess_apply(A, u, yd);
    }
    float xw[3] = {0.f, 0.f, 0.f};
    if (a.gbar) {
      // stencil-weight term of x_p: -sum_i (lambda_i . g_c + v_i . y) grad w_ip
      float gw[3];
      lane_weight_grad(g, xp, lane, gw);
      double lam[3];
      lambda_at(vXh, vXl, ci, lam);
      const float4 vi = lane < 27 ? __ldg(a.G.v + ln.node) : zero4;
      double gc[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) gc[r] = (double)A.dN * A.n[r] + (double)A.cs * A.ut[r];
      const float term = (float)(lam[0] * gc[0] + lam[1] * gc[1] + lam[2] * gc[2] +
                                 (double)vi.x * yd[0] + (double)vi.y * yd[1] + (double)vi.z * yd[2]);
#pragma unroll
      for (int r = 0; r < 3; ++r) xw[r] = warp_sum(-term * gw[r]);
    }
    if (lane == 0 && a.gbar) {
      const int slot = a.slot_of[a.C.id[p].x];
      const float vp[3] = {a.P.v(0)[slot], a.P.v(1)[slot], a.P.v(2)[slot]};
      float xb[3], vb[3];
      double rot[3], wdir[3];
      contact_input_adjoint(A, s_body[body], xp, a.C.vc[p], a.C.bias[p], vp, a.h, u, yd, xb, vb,
                            rot, wdir);
      const size_t np = (size_t)a.n_particles;
      // the moment arm of the body's moment: L = sum r x dl_c, r = x_p - p
      float arm[3] = {0.f, 0.f, 0.f};
      if (a.body_gbar) {
        const double* lb = a.body_gbar + 6 * body + 3;
        const double gc[3] = {(double)A.dN * A.n[0] + (double)A.cs * A.ut[0],
                              (double)A.dN * A.n[1] + (double)A.cs * A.ut[1],
                              (double)A.dN * A.n[2] + (double)A.cs * A.ut[2]};
        arm[0] = (float)(gc[1] * lb[2] - gc[2] * lb[1]);
        arm[1] = (float)(gc[2] * lb[0] - gc[0] * lb[2]);
        arm[2] = (float)(gc[0] * lb[1] - gc[1] * lb[0]);
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        atomicAdd(a.pbar + r * np + slot, xb[r] + xw[r] + arm[r]);
        atomicAdd(&s_bb[body][7 + r], -(double)arm[r]);
        atomicAdd(a.pbar + (3 + r) * np + slot, vb[r]);
        // the contact geometry depends on x_p - p_body: dL/dp = -(its part of
        // dL/dx_p); the body velocity enters n0 through -v: dL/dv gets -vbar
        atomicAdd(&s_bb[body][7 + r], -(double)xb[r]);
        atomicAdd(&s_bb[body][10 + r], -(double)vb[r]);
        atomicAdd(&s_bb[body][13 + r], rot[r]);
        atomicAdd(&s_bb[body][16 + r], wdir[r]);
      }
    }
    if (lane == 0) {
      const float y[3] = {(float)yd[0], (float)yd[1], (float)yd[2]};
      const float mub = (float)(-(double)A.n0_s * ((double)A.ut[0] * u[0] + (double)A.ut[1] * u[1] +
                                                   (double)A.ut[2] * u[2]));
      if (a.contact_bar && p < a.contact_cap) {  // caller memory: 4-byte alignment only
        float* o = a.contact_bar + 4 * (size_t)p;
        o[0] = y[0]; o[1] = y[1]; o[2] = y[2]; o[3] = mub;
      }
      const DevBody& bd = s_body[body];
      const double r0 = (double)xp.x - bd.p[0], r1 = (double)xp.y - bd.p[1], r2 = (double)xp.z - bd.p[2];
      atomicAdd(&s_bb[body][0], yd[0]);
      atomicAdd(&s_bb[body][1], yd[1]);
      atomicAdd(&s_bb[body][2], yd[2]);
      atomicAdd(&s_bb[body][3], r1 * yd[2] - r2 * yd[1]);
      atomicAdd(&s_bb[body][4], r2 * yd[0] - r0 * yd[2]);
      atomicAdd(&s_bb[body][5], r0 * yd[1] - r1 * yd[0]);
      atomicAdd(&s_bb[body][6], (double)mub);
    }
  }
  __syncthreads();
  for (int i = tid; i < a.nb * kAdjBodySlots; i += kThreads) {
    const double v = (&s_bb[0][0])[i];
    if (v != 0.0) atomicAdd(a.body_bar + i, v);
  }
  if (!grid_sync(B)) return;
  // ---- dL/dv* on the contact nodes (into q)
  for (int t = gtid; t < ncn; t += gstride) {
    const float4 L1 = vL1[t];
    double* d = acc64 + 4 * (size_t)t;
    const double y[3] = {__ldcg(d), __ldcg(d + 1), __ldcg(d + 2)};
    d[0] = d[1] = d[2] = 0.0;
    float4 o;
    if (L1.z != 0.f) {
      const float4 h = vXh[t], l = vXl[t];
      const double m = (double)L1.w;
      const double lam[3] = {(double)h.x + (double)l.x, (double)h.y + (double)l.y,
                             (double)h.z + (double)l.z};
      o = make_float4((float)(m * lam[0]), (float)(m * lam[1]), (float)(m * lam[2]), 0.f);
      if (a.gbar) {
        // the mass in M (v - v*) of Eq. (9): mbar = -lambda . (v - v*)
        const int node = a.G.cnodes[t];
        const float4 v = a.G.v[node], vs = a.G.vs[node];
        o.w = (float)(-(lam[0] * (double)(v.x - vs.x) + lam[1] * (double)(v.y - vs.y) +
                        lam[2] * (double)(v.z - vs.z)));
      }
    } else {
      const float4 b = vRhs[t];
      o = make_float4((float)((double)b.x - y[0]), (float)((double)b.y - y[1]),
                      (float)((double)b.z - y[2]), 0.f);
    }
    vQ[t] = o;
    if (a.gbar) a.gbar[a.G.cnodes[t]] = o;
  }
  if (!grid_sync(B)) return;
  for (int i = gtid; i < a.n_in; i += gstride) {
    const int node = node_of_id(a.ids[i]);
    float o[3] = {0.f, 0.f, 0.f};
    if (node >= 0) {
      const int ci = __ldcg(a.G.cflag + node) - 1;
      if (ci >= 0) {
        const float4 q = __ldcg(vQ + ci);
        o[0] = q.x; o[1] = q.y; o[2] = q.z;
      } else {
        o[0] = a.vbar[3 * i]; o[1] = a.vbar[3 * i + 1]; o[2] = a.vbar[3 * i + 2];
      }
    }
    a.vstar_bar[3 * i] = o[0];
    a.vstar_bar[3 * i + 1] = o[1];
    a.vstar_bar[3 * i + 2] = o[2];
  }
  if (!grid_sync(B)) return;
  // release the node flags
  for (int t = gtid; t < ncn; t += gstride) a.G.cflag[a.G.cnodes[t]] = 0;
  if (gtid == 0) {
    a.out[0] = (float)it;
    a.out[1] = rz_ref > 0.f ? sqrtf(fmaxf(rz_true, 0.f) / rz_ref) : 0.f;
    a.out[2] = (float)nc;
    a.out[3] = (float)ncn;
  }
}
}  // namespace

int solve_block_size() { return kThreads; }
const void* solve_kernel_ptr() { return reinterpret_cast<const void*>(&k_solve<false>); }
// the line-search cache, then each thread's first contact stencil (node, weight)
size_t solve_dynamic_smem() {
  return 3 * sizeof(float4) * kLsCacheSlots + (size_t)kThreads * kGrpNodes * (sizeof(int) + sizeof(float));
}
cudaError_t solve_prepare() {
  cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_solve<false>),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)solve_dynamic_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_solve<true>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_dynamic_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_solve<true>),
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (const void* f : {reinterpret_cast<const void*>(&k_solve_batch<1>),
                        reinterpret_cast<const void*>(&k_solve_batch<2>),
                        reinterpret_cast<const void*>(&k_solve_batch<4>),
                        reinterpret_cast<const void*>(&k_solve_batch<8>)})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_dynamic_smem());
  return e;
}

namespace {
cudaLaunchConfig_t cluster_config(int blocks, cudaLaunchAttribute* attr, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = solve_dynamic_smem();
  cfg.stream = s;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = blocks;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}
}  // namespace

int solve_cluster_blocks() {
  for (int blocks : {16, 8, 4}) {
    cudaLaunchAttribute attr;
    const cudaLaunchConfig_t cfg = cluster_config(blocks, &attr, nullptr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, reinterpret_cast<const void*>(&k_solve<true>),
                                       &cfg) == cudaSuccess &&
        clusters >= 1)
      return blocks;
    cudaGetLastError();
  }
  return 0;
}

cudaError_t launch_solve(const SolveArgs& a, int grid_blocks, int cluster_blocks, cudaStream_t s) {
  SolveArgs args = a;
  if (cluster_blocks > 0 && args.cluster_max > 0) {
    cudaLaunchAttribute attr;
    const cudaLaunchConfig_t cfg = cluster_config(cluster_blocks, &attr, s);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_solve<true>, args);
    if (e != cudaSuccess) return e;
  } else {
    args.cluster_max = 0;
  }
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_solve<false>),
                                     dim3(grid_blocks), dim3(kThreads), params,
                                     solve_dynamic_smem(), s);
}

namespace {
template <int kBlocks>
cudaError_t launch_solve_batch_k(const SolveArgs* args, const int* order, int n_scenes,
                                 cudaStream_t s) {
  if (kBlocks == 1) {
    k_solve_batch<1><<<n_scenes, kThreads, solve_dynamic_smem(), s>>>(args, order);
    return cudaGetLastError();
  }
  cudaLaunchAttribute attr;
  const cudaLaunchConfig_t cfg0 = cluster_config(kBlocks, &attr, s);
  cudaLaunchConfig_t cfg = cfg0;
  cfg.gridDim = dim3(n_scenes * kBlocks);
  cfg.attrs = &attr;
  return cudaLaunchKernelEx(&cfg, k_solve_batch<kBlocks>, args, order);
}
}  // namespace

cudaError_t launch_solve_batch(const SolveArgs* args, const int* order, int n_scenes,
                               int blocks_per_scene, cudaStream_t s) {
  if (n_scenes <= 0) return cudaSuccess;
  switch (blocks_per_scene) {
    case 2: return launch_solve_batch_k<2>(args, order, n_scenes, s);
    case 4: return launch_solve_batch_k<4>(args, order, n_scenes, s);
    case 8: return launch_solve_batch_k<8>(args, order, n_scenes, s);
    default: return launch_solve_batch_k<1>(args, order, n_scenes, s);
  }
}

const void* adjoint_kernel_ptr() { return reinterpret_cast<const void*>(&k_adjoint); }

cudaError_t launch_adjoint(const AdjointArgs& a, int grid_blocks, cudaStream_t s) {
  AdjointArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_adjoint), dim3(grid_blocks),
                                     dim3(kThreads), params, 0, s);
}

}  // namespace mpmcr
