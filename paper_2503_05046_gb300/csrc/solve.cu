// solve.cu -- the contact solve of one substep (Eq. (7)-(8)) by the
// quasi-Newton iteration of Alg. 1 (Sec. IV-C, V-B), entirely on the device.
//
// One cooperative launch runs the whole iteration: all thread blocks are
// co-resident and step through the phases in lockstep, separated by a grid
// barrier whose spin has an iteration limit (on expiry the kernel records
// MPM_ERR_TIMEOUT and every block returns). Per iteration:
//   G  contacts: v_c += alpha dv_c; gradient (3) and Hessian (3x3) of the
//      lagged contact potential at v_c, scattered to the nodes with weights
//      w and w^2 (the 3x3 diagonal blocks of J^T (d2 l_c) J, Eq. (10));
//      nodes: v += alpha dv.
//   N  nodes: g = M (v - v*) + J^T dl_c (Eq. (9)), H = M + contact blocks,
//      stopping norms, dv = -H^-1 g by 3x3 Cholesky; grid sums for the line
//      search, A = dv^T M dv and B = dv^T M (v - v*).
//   C  contacts: dv_c = J dv (a G2P gather) and the first line-search
//      derivatives at alpha = 0 and 1.
//   L  line search: f'(alpha) = B + alpha A + sum_p dl_c . dv_c and f'' are
//      contact-only reductions; Newton steps safeguarded by bisection.
// Every block reads the same reduced sums, so all take the same decisions.
// Scalar sums are accumulated per thread and per warp in FP32, across warps
// and blocks in FP64.
#include <cfloat>

#include "kernels.h"

namespace mpmcr {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kSpinLimit = 1u << 24;  // ~1 s of polling with the back-off below

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ double ld_cg(const double* p) {
  return __ldcg(p);
}

struct Barrier {
  unsigned* bar;  // [0] arrivals, [1] generation
  unsigned n;
  unsigned gen;   // meaningful in thread 0 only
  uint32_t* status;
};

// Returns false if any block gave up waiting (the caller then returns).
__device__ bool grid_sync(Barrier& B) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    unsigned arrived = atomicAdd(&B.bar[0], 1u);
    if (arrived == B.n - 1) {
      atomicExch(&B.bar[0], 0u);
      __threadfence();
      atomicExch(&B.bar[1], B.gen + 1u);
    } else {
      unsigned spins = 0;
      while (ld_acquire(&B.bar[1]) == B.gen) {
        if (++spins > kSpinLimit) {
          atomicOr(B.status, kStTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    B.gen += 1u;
    __threadfence();
    if (*reinterpret_cast<volatile uint32_t*>(B.status) & kStTimeout) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int NV>
__device__ void block_reduce_add(float (&v)[NV], double* dst, double (*s_red)[8]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[w][i] = (double)x;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = lane < kWarps ? s_red[lane][i] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) atomicAdd(dst + i, x);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void gather(const GridDev& g, const float4* __restrict__ f,
                                       const float4& xp, float (&out)[3]) {
  Stencil s;
  stencil(g, xp.x, xp.y, xp.z, s);
  out[0] = out[1] = out[2] = 0.f;
#pragma unroll
  for (int cz = 0; cz < 3; ++cz)
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
      const float wyz = s.w[1][cy] * s.w[2][cz];
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const float w = s.w[0][cx] * wyz;
        const float4 q = __ldcg(f + node_index(g, s.base[0] + cx, s.base[1] + cy, s.base[2] + cz));
        out[0] += w * q.x;
        out[1] += w * q.y;
        out[2] += w * q.z;
      }
    }
}

__device__ __forceinline__ void load_contact(const Contacts& C, int p, float4& xp, float (&n)[3],
                                             float& n0) {
  xp = C.xp[p];
  const float4 q = C.nrm[p];
  n[0] = q.x; n[1] = q.y; n[2] = q.z;
  n0 = q.w;
}

// derivative sums of the line search at alpha for this thread's contacts
__device__ void ls_eval(const SolveArgs& a, const DevBody* s_body, int nc, float alpha,
                        float (&acc)[2]) {
  acc[0] = acc[1] = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nc; p += gridDim.x * blockDim.x) {
    float4 xp; float n[3]; float n0;
    load_contact(a.C, p, xp, n, n0);
    const DevBody& bd = s_body[a.C.id[p].y];
    const float4 vc = a.C.vc[p], dvc = a.C.dvc[p];
    const float u[3] = {vc.x + alpha * dvc.x, vc.y + alpha * dvc.y, vc.z + alpha * dvc.z};
    const float e[3] = {dvc.x, dvc.y, dvc.z};
    ContactLaw L;
    contact_law(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u, L);
    float d1, d2;
    contact_dir(L, n, e, d1, d2);
    acc[0] += d1;
    acc[1] += d2;
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_solve(SolveArgs a) {
  __shared__ DevBody s_body[kMaxBodies];
  __shared__ double s_red[kWarps][8];
  __shared__ float s_imp[kMaxBodies][6];
  const int tid = threadIdx.x;
  for (int i = tid; i < a.nb * (int)(sizeof(DevBody) / 4); i += kThreads)
    reinterpret_cast<float*>(s_body)[i] = reinterpret_cast<const float*>(a.bodies)[i];
  for (int i = tid; i < kMaxBodies * 6; i += kThreads) (&s_imp[0][0])[i] = 0.f;
  const int count = *a.C.count;
  const int nc = count < a.C.cap ? count : a.C.cap;
  const long long n_nodes = (long long)(*a.G.n_act) * kBlockNodes;
  __syncthreads();
  if (nc == 0) return;  // v = v* already (set by the grid update)

  Barrier B{a.bar, gridDim.x, 0u, a.status};
  if (tid == 0) B.gen = ld_acquire(&a.bar[1]);
  const int gtid = blockIdx.x * kThreads + tid;
  const int gstride = gridDim.x * kThreads;
  const GridDev& g = a.g;
  int rslot = 0;
  auto next_slot = [&]() -> double* {
    double* s = a.red + 8 * (rslot & 3);
    if (blockIdx.x == 0 && tid < 8) a.red[8 * ((rslot + 2) & 3) + tid] = 0.0;
    ++rslot;
    return s;
  };

  // v_c = J v + b at v = v* (Alg. 1 initialisation)
  for (int p = gtid; p < nc; p += gstride) {
    float u[3];
    gather(g, a.G.v, a.C.xp[p], u);
    const float4 b = a.C.bias[p];
    a.C.vc[p] = make_float4(u[0] + b.x, u[1] + b.y, u[2] + b.z, 0.f);
  }
  if (!grid_sync(B)) return;

  double alpha = 0.0;
  int it = 0, ls_evals = 0;
  float resid = 0.f;
  for (;;) {
    // ---- G: update by the last step, contact gradient / Hessian blocks
    const float al = (float)alpha;
    for (int p = gtid; p < nc; p += gstride) {
      float4 xp; float n[3]; float n0;
      load_contact(a.C, p, xp, n, n0);
      float4 vc = a.C.vc[p];
      if (it > 0) {
        const float4 dvc = a.C.dvc[p];
        vc.x += al * dvc.x; vc.y += al * dvc.y; vc.z += al * dvc.z;
        a.C.vc[p] = vc;
      }
      const DevBody& bd = s_body[a.C.id[p].y];
      const float u[3] = {vc.x, vc.y, vc.z};
      ContactLaw L;
      contact_law(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u, L);
      float gr[3], H[6];
      contact_grad(L, n, gr);
      contact_hess(L, n, H);
      Stencil s;
      stencil(g, xp.x, xp.y, xp.z, s);
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
          const float wyz = s.w[1][cy] * s.w[2][cz];
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const float w = s.w[0][cx] * wyz, w2 = w * w;
            const int node = node_index(g, s.base[0] + cx, s.base[1] + cy, s.base[2] + cz);
            red_add_v4(a.G.acc0 + node, w * gr[0], w * gr[1], w * gr[2], w2 * H[0]);
            red_add_v4(a.G.acc1 + node, w2 * H[1], w2 * H[2], w2 * H[3], w2 * H[4]);
            red_add_f32(a.G.acc2 + node, w2 * H[5]);
          }
        }
    }
    if (it > 0) {
      for (long long t = gtid; t < n_nodes; t += gstride) {
        const int node = a.G.act[t >> 6] * kBlockNodes + (int)(t & 63);
        float4 v = a.G.v[node];
        const float4 d = a.G.dv[node];
        v.x += al * d.x; v.y += al * d.y; v.z += al * d.z;
        a.G.v[node] = v;
      }
    }
    if (!grid_sync(B)) return;

    // ---- N: gradient, stopping norms, direction, grid line-search sums
    {
      double* slot = next_slot();
      float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // G2, P2, J2, A, B
      for (long long t = gtid; t < n_nodes; t += gstride) {
        const int node = a.G.act[t >> 6] * kBlockNodes + (int)(t & 63);
        const float4 vs = a.G.vs[node];
        const float m = vs.w;
        float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m > 0.f) {
          const float4 v = a.G.v[node];
          // written by other blocks' reductions in this launch: read from L2
          const float4 c0 = __ldcg(a.G.acc0 + node);
          const float4 c1 = __ldcg(a.G.acc1 + node);
          const float c2 = __ldcg(a.G.acc2 + node);
          a.G.acc0[node] = make_float4(0.f, 0.f, 0.f, 0.f);
          a.G.acc1[node] = make_float4(0.f, 0.f, 0.f, 0.f);
          a.G.acc2[node] = 0.f;
          if (v.w == 0.f) {  // free DoF (v.w flags a Dirichlet node)
            const float r0 = v.x - vs.x, r1 = v.y - vs.y, r2 = v.z - vs.z;
            const float g0 = m * r0 + c0.x, g1 = m * r1 + c0.y, g2 = m * r2 + c0.z;
            const float inv_m = 1.0f / m;
            acc[0] += (g0 * g0 + g1 * g1 + g2 * g2) * inv_m;
            acc[1] += m * (v.x * v.x + v.y * v.y + v.z * v.z);
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
        }
        a.G.dv[node] = dv;
      }
      block_reduce_add(acc, slot, s_red);
      if (!grid_sync(B)) return;
      const double G2 = ld_cg(slot + 0), P2 = ld_cg(slot + 1), J2 = ld_cg(slot + 2);
      const double A = ld_cg(slot + 3), Bs = ld_cg(slot + 4);
      const double Gn = sqrt(G2), Pn = sqrt(P2), Jn = sqrt(J2);
      const double mx = Pn > Jn ? Pn : Jn;
      resid = mx > 0.0 ? (float)(Gn / mx) : 0.f;
      if (!(G2 == G2) || !(A == A) || !(Bs == Bs)) {
        if (gtid == 0) atomicOr(a.status, kStNan);
        break;
      }
      if (Gn < a.eps_a + a.eps_r * mx || G2 == 0.0) break;  // converged
      if (it >= a.max_iters) {
        if (gtid == 0) atomicOr(a.status, kStNotConverged);
        break;
      }

      // ---- C: dv_c = J dv and the line-search derivatives at 0 and 1
      double* slot2 = next_slot();
      float lacc[3] = {0.f, 0.f, 0.f};  // S1(0), S1(1), S2(1)
      for (int p = gtid; p < nc; p += gstride) {
        float4 xp; float n[3]; float n0;
        load_contact(a.C, p, xp, n, n0);
        float e[3];
        gather(g, a.G.dv, xp, e);
        a.C.dvc[p] = make_float4(e[0], e[1], e[2], 0.f);
        const float4 vc = a.C.vc[p];
        const DevBody& bd = s_body[a.C.id[p].y];
        ContactLaw L;
        float d1, d2;
        const float u0[3] = {vc.x, vc.y, vc.z};
        contact_law(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u0, L);
        contact_dir(L, n, e, d1, d2);
        lacc[0] += d1;
        const float u1[3] = {vc.x + e[0], vc.y + e[1], vc.z + e[2]};
        contact_law(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u1, L);
        contact_dir(L, n, e, d1, d2);
        lacc[1] += d1;
        lacc[2] += d2;
      }
      block_reduce_add(lacc, slot2, s_red);
      if (!grid_sync(B)) return;
      ls_evals += 2;
      const double fp0 = Bs + ld_cg(slot2 + 0);
      double lo = 0.0, hi = 1.0;
      double d1 = Bs + A + ld_cg(slot2 + 1);
      double d2 = A + ld_cg(slot2 + 2);
      if (!(fp0 < 0.0)) {  // no descent left at working precision
        alpha = 0.0;
        break;
      }
      bool failed = false;
      while (d1 < 0.0) {  // expand the bracket
        lo = hi;
        hi *= 2.0;
        if (hi > 1024.0) { failed = true; break; }
        double* sl = next_slot();
        float e2[2];
        ls_eval(a, s_body, nc, (float)hi, e2);
        block_reduce_add(e2, sl, s_red);
        if (!grid_sync(B)) return;
        ++ls_evals;
        d1 = Bs + hi * A + ld_cg(sl);
        d2 = A + ld_cg(sl + 1);
      }
      if (failed) {
        if (gtid == 0) atomicOr(a.status, kStLineSearch);
        alpha = lo;
        ++it;
        continue;
      }
      const double tol = (double)a.ls_rel_tol * fabs(fp0);
      double x = hi, prev = DBL_MAX;
      for (int k = 0; k < a.ls_max_iters; ++k) {
        if (fabs(d1) <= tol) break;
        if (d1 < 0.0) lo = x; else hi = x;
        const double xn = x - d1 / d2;
        const bool newton = d2 > 0.0 && xn > lo && xn < hi && fabs(d1) <= 0.5 * prev;
        prev = fabs(d1);
        x = newton ? xn : 0.5 * (lo + hi);
        double* sl = next_slot();
        float e2[2];
        ls_eval(a, s_body, nc, (float)x, e2);
        block_reduce_add(e2, sl, s_red);
        if (!grid_sync(B)) return;
        ++ls_evals;
        d1 = Bs + x * A + ld_cg(sl);
        d2 = A + ld_cg(sl + 1);
        if (hi - lo <= 1e-7 * hi) break;
      }
      alpha = x;
      ++it;
    }
  }

  // ---- impulses at the solution: gamma = -dl_c/dv_c on the particle; the
  // body receives -gamma and its moment about the body origin (Eq. (3))
  for (int p = gtid; p < nc; p += gstride) {
    float4 xp; float n[3]; float n0;
    load_contact(a.C, p, xp, n, n0);
    const int b = a.C.id[p].y;
    const DevBody& bd = s_body[b];
    const float4 vc = a.C.vc[p];
    const float u[3] = {vc.x, vc.y, vc.z};
    ContactLaw L;
    contact_law(xp.w, n0, bd.mu, bd.k, bd.d, a.h, a.eps_s, n, u, L);
    float gr[3];
    contact_grad(L, n, gr);
    a.C.gamma[p] = make_float4(-gr[0], -gr[1], -gr[2], 0.f);
    const float r0 = xp.x - bd.p[0], r1 = xp.y - bd.p[1], r2 = xp.z - bd.p[2];
    atomicAdd(&s_imp[b][0], gr[0]);
    atomicAdd(&s_imp[b][1], gr[1]);
    atomicAdd(&s_imp[b][2], gr[2]);
    atomicAdd(&s_imp[b][3], r1 * gr[2] - r2 * gr[1]);
    atomicAdd(&s_imp[b][4], r2 * gr[0] - r0 * gr[2]);
    atomicAdd(&s_imp[b][5], r0 * gr[1] - r1 * gr[0]);
  }
  __syncthreads();
  for (int i = tid; i < a.nb * 6; i += kThreads) {
    const float v = (&s_imp[0][0])[i];
    if (v != 0.f) atomicAdd(a.impulses + i, (double)v);
  }
  if (gtid == 0) {
    atomicAdd(&a.stats->iters_total, it);
    atomicMax(&a.stats->iters_max, it);
    atomicAdd(&a.stats->ls_evals_total, ls_evals);
    atomicMax(reinterpret_cast<int*>(&a.stats->residual_max), __float_as_int(resid));
  }
}

}  // namespace

int solve_block_size() { return kThreads; }
const void* solve_kernel_ptr() { return reinterpret_cast<const void*>(&k_solve); }

cudaError_t launch_solve(const SolveArgs& a, int grid_blocks, cudaStream_t s) {
  SolveArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_solve), dim3(grid_blocks),
                                     dim3(kThreads), params, 0, s);
}

}  // namespace mpmcr
