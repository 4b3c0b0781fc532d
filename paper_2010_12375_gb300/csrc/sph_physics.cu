// Pair-interaction kernels and time-step control of the WCSPH hot path.
//
//   k_density              Eq. eqrhosum / Eq. eqrhosumnosurface (once per advection step)
//   k_viscous              Eq. eqviscous (once per advection step, fluid pairs)
//   k_dt_advection         Eq. dt-advection (one thread per instance, FP64)
//   k_dt_acoustic          Eq. dt-relax clamped to the advection step (one thread per instance)
//   (the acoustic-substep relaxation kernels live in sph_relax.cuh)
//
// Conventions: r_ij = r_i - r_j, e_ij = -r_ij/|r_ij| points from i to j, and
// grad_i W_ij = (dW/dr) r_ij/|r_ij|. Interface states of the low-dissipation
// solver: U* = (U_L+U_R)/2 + (P_L-P_R)/(2 rho_bar c0),
// P* = (P_L+P_R)/2 + rho_bar c0 beta (U_L-U_R)/2, beta = min(3 max(U_L-U_R,0)/c0, 1).
// One thread per fluid particle walks its frozen neighbour row (column-major
// ELL, so a warp's 32 index loads per row position are one 128-byte line) and
// recomputes the pair geometry from the current positions; pairs at or beyond
// 2h, or at zero distance, contribute nothing.
#include <cmath>

#include "sph_ctrl.cuh"
#include "sph_kernels.h"

namespace sph {

namespace {

constexpr int kBlock = 256;

inline unsigned grid_for(int64_t n, int block = kBlock) {
  return (unsigned)((n + block - 1) / block);
}

__device__ __forceinline__ void raise_error(Global* g, int bit, long long idx) {
  int old = atomicOr(&g->err, bit);
  if (old == 0) g->bad_index = idx;
}

__device__ __forceinline__ int inst_index(const int* inst_of, int64_t i) {
  return inst_of ? inst_of[i] : 0;
}

// Block-wide max of |v|^2 into the instance's slot: one atomic per block when the
// whole block belongs to one instance, else one per lane.
__device__ __forceinline__ void reduce_vmax(float v2, bool valid, int k, bool uniform_block,
                                            Ctrl* ctrl) {
  __shared__ float red[kBlock / 32];
  if (!uniform_block) {
    if (valid) atomicMax(&ctrl[k].vmax2, __float_as_uint(v2));
    return;
  }
  float m = valid ? v2 : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(&ctrl[k].vmax2, __float_as_uint(m));
  }
}

__device__ __forceinline__ bool block_one_instance(const int* inst_of, int64_t n, int* k_out) {
  int64_t first = (int64_t)blockIdx.x * blockDim.x;
  int64_t last = min(first + (int64_t)blockDim.x, n) - 1;
  int a = inst_index(inst_of, first), b = inst_index(inst_of, last);
  *k_out = a;
  return a == b;
}

// ---------------------------------------------------------------- import / export ----
template <int D>
__global__ void k_import(int64_t i0, int64_t n, const double* __restrict__ pos, const double* __restrict__ vel,
                         const double* __restrict__ rho, const double* __restrict__ drho,
                         const int* __restrict__ inst_of, const Inst* __restrict__ inst,
                         int4* __restrict__ P, float4* __restrict__ V, Global* g) {
  int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // rows [i0, n)
  if (i >= n) return;
  const Inst& I = inst[inst_index(inst_of, i)];
  int q[3] = {0, 0, 0};
  float v[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double s = (pos[i * D + a] - I.lo[a]) / I.dq_d;
    double lim = 2147483000.0;
    if (!(s > -lim && s < lim)) {          // also catches NaN
      raise_error(g, ERR_DOMAIN, i);
      s = 0.0;
    }
    int qa = __double2int_rn(s);
    if (I.period[a]) {
      qa %= I.period[a];
      if (qa < 0) qa += I.period[a];
    }
    q[a] = qa;
    v[a] = (float)vel[i * D + a];
  }
  float dev = (float)(rho[i] - I.rho0_d);
  float dr = drho ? (float)drho[i] : 0.0f;
  P[i] = make_int4(q[0], q[1], q[2], f2i(dev));
  V[i] = make_float4(v[0], v[1], v[2], dr);
}

template <int D>
__global__ void k_import_walls(int64_t n, const double* __restrict__ pos, const double* __restrict__ nrm,
                               const double* __restrict__ vol, const int* __restrict__ inst_of,
                               const Inst* __restrict__ inst, int4* __restrict__ P,
                               float4* __restrict__ N, Global* g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_index(inst_of, i)];
  int q[3] = {0, 0, 0};
  float nv[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double s = (pos[i * D + a] - I.lo[a]) / I.dq_d;
    if (!(s > -2147483000.0 && s < 2147483000.0)) {
      raise_error(g, ERR_DOMAIN, i);
      s = 0.0;
    }
    int qa = __double2int_rn(s);
    if (I.period[a]) {
      qa %= I.period[a];
      if (qa < 0) qa += I.period[a];
    }
    q[a] = qa;
    nv[a] = (float)nrm[i * D + a];
  }
  P[i] = make_int4(q[0], q[1], q[2], f2i((float)vol[i]));
  N[i] = make_float4(nv[0], nv[1], nv[2], 0.0f);
}

template <int D>
__global__ void k_export(int64_t n, const int4* __restrict__ P, const float4* __restrict__ V,
                         const int* __restrict__ id, const int* __restrict__ inst_of,
                         const Inst* __restrict__ inst, double* __restrict__ pos,
                         double* __restrict__ vel, double* __restrict__ rho,
                         double* __restrict__ drho) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_index(inst_of, i)];
  int4 p = P[i];
  float4 v = V[i];
  int64_t row = id[i];
  int q[3] = {p.x, p.y, p.z};
  float vv[3] = {v.x, v.y, v.z};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (pos) pos[row * D + a] = I.lo[a] + (double)q[a] * I.dq_d;
    if (vel) vel[row * D + a] = (double)vv[a];
  }
  if (rho) rho[row] = I.rho0_d + (double)i2f(p.w);
  if (drho) drho[row] = (double)v.w;
}

template <int D>
__global__ void k_export_acc(int64_t n, const float4* __restrict__ A, const int* __restrict__ id,
                             double* __restrict__ acc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 a = A[i];
  int64_t row = id[i];
  acc[row * D + 0] = a.x;
  acc[row * D + 1] = a.y;
  if (D == 3) acc[row * D + 2] = a.z;
}

__global__ void k_export_neighbours(int64_t n, int cap, const int* __restrict__ nbr,
                                    const uint32_t* __restrict__ nbc, const int* __restrict__ id,
                                    const int* __restrict__ wid, int stride, int32_t* __restrict__ fc,
                                    int32_t* __restrict__ wc, int32_t* __restrict__ fids,
                                    int32_t* __restrict__ wids) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c = nbc[i];
  int nf = (int)(c & 0xffffu), nw = (int)(c >> 16);
  int64_t row = id[i];
  fc[row] = nf;
  wc[row] = nw;
  for (int k = 0; k < nf; ++k) fids[row * stride + k] = id[nbr[slot_index(n, i, k)]];
  const int w0 = wall_slot0(nf);
  for (int k = 0; k < nw; ++k) wids[row * stride + k] = wid[nbr[slot_index(n, i, w0 + k)]];
}

__global__ void k_pair_count(int64_t n, const uint32_t* __restrict__ nbc, unsigned long long* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long f = 0, w = 0;
  if (i < n) {
    f = nbc[i] & 0xffffu;
    w = nbc[i] >> 16;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(0xffffffffu, f, o);
    w += __shfl_xor_sync(0xffffffffu, w, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], f);
    atomicAdd(&out[1], w);
  }
}

// ---------------------------------------------------------------- reductions / steps -
template <int D>
__global__ void k_vmax(int64_t n, const float4* __restrict__ V, const int* __restrict__ inst_of,
                       Ctrl* ctrl) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int k;
  bool uni = block_one_instance(inst_of, n, &k);
  float v2 = 0.f;
  bool valid = i < n;
  if (valid) {
    float4 v = V[i];
    v2 = v.x * v.x + v.y * v.y + (D == 3 ? v.z * v.z : 0.f);
    if (!uni) k = inst_index(inst_of, i);
  }
  reduce_vmax(v2, valid, k, uni, ctrl);
}

__global__ void k_reset_vmax(int n_inst, Ctrl* ctrl) {
  for (int k = threadIdx.x; k < n_inst; k += blockDim.x) ctrl[k].vmax2 = 0u;
}

// Eq. dt-advection: Dt_ad = CFL_ad min(h / max(|v|max, U_ref), h^2 / nu).
__global__ void k_dt_advection(int n_inst, const Inst* __restrict__ inst, Ctrl* ctrl, Global* g) {
  for (int k = threadIdx.x; k < n_inst; k += blockDim.x) {
    const Inst& I = inst[k];
    Ctrl& C = ctrl[k];
    double vmax = sqrt((double)__uint_as_float(C.vmax2));
    double dt = I.h_d / fmax(vmax, I.u_ref);
    if (I.nu > 0.0) dt = fmin(dt, I.h_d * I.h_d / I.nu);
    C.dt_ad = I.cfl_ad * dt;
    C.tau = 0.0;
    C.done = 0;
    C.dt = 0.0;
    C.sub_in_step = 0;
    C.adv_steps += 1;
  }
  if (threadIdx.x == 0) g->active = 1;
}

// Eq. dt-relax, clamped to the remainder of the advection step (block body in
// sph_ctrl.cuh). Sets the condition of the device-side substep loop when launched inside
// a graph.
__global__ void k_dt_acoustic(int n_inst, const Inst* __restrict__ inst, Ctrl* ctrl, Global* g,
                              cudaGraphConditionalHandle cond, int use_cond, const double* dt_cap) {
  const int any = dt_acoustic_block(n_inst, inst, ctrl, g, dt_cap);
  if (threadIdx.x == 0) {
    g->active = any;
    g->substeps += 1;
    if (use_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

// ---------------------------------------------------------------- density -------------
// W of two pairs at once from their packed squared distances; lanes with mask 0 add 0.
__device__ __forceinline__ float2 kernel_W2(float2 r2, float inv_h, float w_a) {
  const float2 q = mul2(mul2(r2, rsqrt2(fma2(r2, f2(1.0f), f2(1e-30f)))), f2(inv_h));
  const float2 t = max2(fma2(q, f2(-0.5f), f2(1.0f)), 0.0f);
  const float2 t2 = mul2(t, t);
  return mul2(mul2(f2(w_a), mul2(t2, t2)), fma2(q, f2(2.0f), f2(1.0f)));
}

template <int D, bool PER>
__device__ __forceinline__ float2 pair_r2(const int4& p, const int4& a, const int4& b, const Inst& I) {
  const float2 M = f2(-kMagic), DQ = f2(I.dq);
  const float2 dx = mul2(add2(make_float2(biased_diff<PER>(p.x, a.x, I.period[0]), biased_diff<PER>(p.x, b.x, I.period[0])), M), DQ);
  const float2 dy = mul2(add2(make_float2(biased_diff<PER>(p.y, a.y, I.period[1]), biased_diff<PER>(p.y, b.y, I.period[1])), M), DQ);
  float2 r2 = fma2(dx, dx, mul2(dy, dy));
  if (D == 3) {
    const float2 dz = mul2(add2(make_float2(biased_diff<PER>(p.z, a.z, I.period[2]), biased_diff<PER>(p.z, b.z, I.period[2])), M), DQ);
    r2 = fma2(dz, dz, r2);
  }
  return r2;
}

// Eq. eqrhosum / Eq. eqrhosumnosurface: rho = rho0 sum W / sum W0 (with max(rho*, .) for a
// free surface), sum over self, fluid and wall neighbours. The Kahan sum starts from
// W(0) - sumW0 so it holds the deviation rho/rho0 - 1 with its own relative precision.
template <int D, bool PER>
__global__ void __launch_bounds__(kBlock)
k_density(int64_t n, int4* P, const int* __restrict__ inst_of, const Inst* __restrict__ inst,
          const int* __restrict__ nbr, const uint32_t* __restrict__ nbc, const int4* __restrict__ WP) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_index(inst_of, i)];
  const int4 pi = P[i];
  const uint32_t c = nbc[i];
  const int nf = (int)(c & 0xffffu), nw = (int)(c >> 16);
  float2 s = make_float2(I.sig_hi, 0.0f), nc = f2(0.0f);
  kahan2(s, nc, make_float2(I.sig_lo, 0.0f), f2(1.0f));
  const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
  const int nq = (nf + 3) >> 2;
  int4 nxt = nq ? nb4[i] : make_int4(0, 0, 0, 0);
  for (int q = 0; q < nq; ++q) {
    const int4 cq = nxt;
    if (q + 1 < nq) nxt = nb4[(int64_t)(q + 1) * n + i];   // next quad in flight
    const int sl = q << 2;
    const int j1 = sl + 1 < nf ? cq.y : cq.x, j2 = sl + 2 < nf ? cq.z : cq.x, j3 = sl + 3 < nf ? cq.w : cq.x;
    const int4 a0 = P[cq.x], a1 = P[j1], a2 = P[j2], a3 = P[j3];
    const float2 m01 = make_float2(1.0f, sl + 1 < nf ? 1.0f : 0.0f);
    const float2 m23 = make_float2(sl + 2 < nf ? 1.0f : 0.0f, sl + 3 < nf ? 1.0f : 0.0f);
    kahan2(s, nc, kernel_W2(pair_r2<D, PER>(pi, a0, a1, I), I.inv_h, I.w_a), m01);
    kahan2(s, nc, kernel_W2(pair_r2<D, PER>(pi, a2, a3, I), I.inv_h, I.w_a), m23);
  }
  const int q0 = wall_slot0(nf) >> 2, nwq = (nw + 3) >> 2;
  for (int q = 0; q < nwq; ++q) {
    const int4 cq = nb4[(int64_t)(q0 + q) * n + i];
    const int sl = q << 2;
    const int w1 = sl + 1 < nw ? cq.y : cq.x, w2 = sl + 2 < nw ? cq.z : cq.x, w3 = sl + 3 < nw ? cq.w : cq.x;
    const int4 a0 = WP[cq.x], a1 = WP[w1], a2 = WP[w2], a3 = WP[w3];
    const float2 m01 = make_float2(1.0f, sl + 1 < nw ? 1.0f : 0.0f);
    const float2 m23 = make_float2(sl + 2 < nw ? 1.0f : 0.0f, sl + 3 < nw ? 1.0f : 0.0f);
    kahan2(s, nc, kernel_W2(pair_r2<D, PER>(pi, a0, a1, I), I.inv_h, I.w_a), m01);
    kahan2(s, nc, kernel_W2(pair_r2<D, PER>(pi, a2, a3, I), I.inv_h, I.w_a), m23);
  }
  float dev = I.rho0_over_sigma0 * ((s.x + nc.x) + (s.y + nc.y));   // rho0 sumW/sumW0 - rho0
  if (I.free_surface) dev = fmaxf(i2f(pi.w), dev);
  reinterpret_cast<int*>(P + i)[3] = f2i(dev);        // only .w changes; others read .xyz
}

template <int D>
__global__ void __launch_bounds__(kBlock)
k_viscous(int64_t n, const int4* __restrict__ P, const float4* __restrict__ V,
          const float* __restrict__ mass, const int* __restrict__ inst_of,
          const Inst* __restrict__ inst, const int* __restrict__ nbr,
          const uint32_t* __restrict__ nbc, float4* __restrict__ acc_prior) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_index(inst_of, i)];
  const int4 pi = P[i];
  const float4 vi = V[i];
  float rho_i = I.rho0 + i2f(pi.w);
  int nf = (int)(nbc[i] & 0xffffu);
  float ax = 0.f, ay = 0.f, az = 0.f;
  if (I.eta > 0.0f) {
    for (int k = 0; k < nf; ++k) {
      int j = nbr[slot_index(n, i, k)];
      const int4 pj = P[j];
      const float4 vj = V[j];
      float dx = (float)wrap_diff(pi.x - pj.x, I.period[0]) * I.dq;
      float dy = (float)wrap_diff(pi.y - pj.y, I.period[1]) * I.dq;
      float r2 = dx * dx + dy * dy;
      if (D == 3) {
        float dz = (float)wrap_diff(pi.z - pj.z, I.period[2]) * I.dq;
        r2 += dz * dz;
      }
      if (!(r2 < I.four_h2) || r2 == 0.0f) continue;
      float fw = kernel_dW_over_r(sqrtf(r2), I);            // (dW/dr)/r
      float mj = mass ? mass[j] : I.mass;
      float f = mj / (I.rho0 + i2f(pj.w)) * fw;
      ax += f * (vi.x - vj.x);
      ay += f * (vi.y - vj.y);
      if (D == 3) az += f * (vi.z - vj.z);
    }
  }
  float s = 2.0f * I.eta / rho_i;
  acc_prior[i] = make_float4(s * ax, s * ay, s * az, 0.0f);
}

}  // namespace

// ---------------------------------------------------------------- launchers -----------
#define SPH_DIM_LAUNCH(b, kern, grid, block, stream, ...)                          \
  do {                                                                             \
    if ((b).dim == 2) kern<2><<<grid, block, 0, stream>>>(__VA_ARGS__);            \
    else kern<3><<<grid, block, 0, stream>>>(__VA_ARGS__);                         \
  } while (0)

void launch_import(const Buffers& b, const double* pos, const double* vel, const double* rho,
                   const double* drho, cudaStream_t s, int64_t i0, int64_t i1) {
  if (i1 < 0) i1 = b.n;
  if (i1 <= i0) return;
  SPH_DIM_LAUNCH(b, k_import, grid_for(i1 - i0), kBlock, s, i0, i1, pos, vel, rho, drho, b.inst_of, b.inst,
                 b.PS, b.VS, b.glob);
}

void launch_import_walls(const Buffers& b, const double* pos, const double* nrm, const double* vol,
                         cudaStream_t s) {
  if (b.nw == 0) return;
  SPH_DIM_LAUNCH(b, k_import_walls, grid_for(b.nw), kBlock, s, b.nw, pos, nrm, vol, b.winst_of, b.inst,
                 b.WP, b.WN, b.glob);
}

void launch_export(const Buffers& b, double* pos, double* vel, double* rho, double* drho,
                   cudaStream_t s) {
  if (b.n == 0) return;
  SPH_DIM_LAUNCH(b, k_export, grid_for(b.n), kBlock, s, b.n, b.PS, b.VS, b.id, b.inst_of, b.inst, pos,
                 vel, rho, drho);
}

void launch_export_acc(const Buffers& b, double* acc, cudaStream_t s) {
  if (b.n == 0 || !b.acc_keep) return;
  SPH_DIM_LAUNCH(b, k_export_acc, grid_for(b.n), kBlock, s, b.n, b.acc_keep, b.id, acc);
}

void launch_export_neighbours(const Buffers& b, int32_t* fc, int32_t* wc, int32_t* fids,
                              int32_t* wids, int32_t stride, cudaStream_t s) {
  if (b.n == 0) return;
  k_export_neighbours<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.cap, b.nbr, b.nbc, b.id, b.wid, stride,
                                                        fc, wc, fids, wids);
}

void launch_pair_count(const Buffers& b, unsigned long long* out2, cudaStream_t s) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), s);
  if (b.n == 0) return;
  k_pair_count<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.nbc, out2);
}

void launch_vmax(const Buffers& b, cudaStream_t s, int64_t* launches) {
  k_reset_vmax<<<1, 256, 0, s>>>(b.n_inst, b.ctrl);
  ++*launches;
  if (b.n == 0) return;
  SPH_DIM_LAUNCH(b, k_vmax, grid_for(b.n), kBlock, s, b.n, b.VS, b.inst_of, b.ctrl);
  ++*launches;
}

void launch_dt_advection(const Buffers& b, cudaStream_t s, int64_t* launches) {
  k_dt_advection<<<1, 256, 0, s>>>(b.n_inst, b.inst, b.ctrl, b.glob);
  ++*launches;
}

void launch_density(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  auto kern = b.dim == 2 ? (b.any_periodic ? k_density<2, true> : k_density<2, false>)
                         : (b.any_periodic ? k_density<3, true> : k_density<3, false>);
  kern<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.PS, b.inst_of, b.inst, b.nbr, b.nbc, b.WP);
  ++*launches;
}

void launch_viscous(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0 || !b.acc_prior) return;
  SPH_DIM_LAUNCH(b, k_viscous, grid_for(b.n), kBlock, s, b.n, b.PS, b.VS, b.mass, b.inst_of, b.inst,
                 b.nbr, b.nbc, b.acc_prior);
  ++*launches;
}

void launch_dt_acoustic(const Buffers& b, cudaStream_t s, cudaGraphConditionalHandle cond,
                        bool use_cond, int64_t* launches) {
  k_dt_acoustic<<<1, 256, 0, s>>>(b.n_inst, b.inst, b.ctrl, b.glob, cond, use_cond ? 1 : 0, b.dt_cap);
  ++*launches;
}

}  // namespace sph
