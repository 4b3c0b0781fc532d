// Acoustic-substep kernels of the position-based Verlet scheme (the hot loop).
//
//   k_pressure_relaxation  Eq. verlet-first-half (rho, r to n+1/2), Eq. eqeos,
//                          Eq. riemannsph momentum with P* of the low-dissipation
//                          solver, wall pairs by the one-sided problem of
//                          Eqs. eqriepartial / eqrienoslip / eqriepright,
//                          Eq. verlet-first-mediate (v to n+1)
//   k_density_relaxation   Eq. verlet-first-final: r to n+1 with v^{n+1}, then
//                          Eq. riemannsph continuity with U*, rho to n+1
//
// r_ij = r_i - r_j, e_ij = -r_ij/|r_ij|, grad_i W_ij = (dW/dr) r_ij/|r_ij|;
// U_L = v_i.e_ij, U_R = v_j.e_ij, U* = (U_L+U_R)/2 + (P_L-P_R)/(2 rho_bar c0),
// P* = (P_L+P_R)/2 + rho_bar c0 beta (U_L-U_R)/2, beta = min(3 max(U_L-U_R,0)/c0, 1).
//
// One thread per fluid particle walks its frozen neighbour row two entries at a
// time: the two pairs occupy the .x and .y lanes of packed FP32 instructions
// (__ffma2_rn and friends), which halves the instruction count of the pair
// arithmetic. An odd row is padded with the particle itself, a pair at zero
// distance whose contribution is exactly zero. Pairs that drifted past 2h get
// t = max(1 - q/2, 0) = 0 and contribute nothing, with no branch. Sums are
// Kahan-compensated per lane and the two lanes are added at the end.
#include "sph_kernels.h"

namespace sph {

namespace {

constexpr int kBlock = 256;
constexpr float kTinyR2 = 1e-30f;     // keeps rsqrt finite for a pair at zero distance

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

__device__ __forceinline__ bool block_one_instance(const int* inst_of, int64_t n, int* k_out) {
  int64_t first = (int64_t)blockIdx.x * blockDim.x;
  int64_t last = min(first + (int64_t)blockDim.x, n) - 1;
  int a = inst_index(inst_of, first), b = inst_index(inst_of, last);
  *k_out = a;
  return a == b;
}

__device__ __forceinline__ void reduce_vmax(float v2, bool valid, int k, bool uniform_block, Ctrl* ctrl) {
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

// Per-pair kernel factor (dW/dr)/r and |r| from the packed pair vector.
struct Geo2 {
  float2 inv_r, r, fw;
};

__device__ __forceinline__ Geo2 geometry2(float2 rx, float2 ry, float2 rz, float inv_h, float dwr) {
  Geo2 g;
  float2 r2 = fma2(rx, rx, fma2(ry, ry, fma2(rz, rz, f2(kTinyR2))));
  g.inv_r = rsqrt2(r2);
  g.r = mul2(r2, g.inv_r);
  float2 t = max2(fma2(g.r, f2(-0.5f * inv_h), f2(1.0f)), 0.0f);   // 1 - q/2, 0 beyond 2h
  g.fw = mul2(f2(dwr), mul2(mul2(t, t), t));                       // -5 alpha/h^2 (1-q/2)^3
  return g;
}

// ---------------------------------------------------------------- pressure relaxation --
template <int D, bool PER>
__global__ void __launch_bounds__(kBlock, 2)
k_pressure_relaxation(int64_t n, const int4* __restrict__ PS, const float4* __restrict__ VS,
                      int4* __restrict__ PH, float4* __restrict__ VH,
                      const float* __restrict__ mass, const int* __restrict__ inst_of,
                      const Inst* __restrict__ inst, Ctrl* ctrl, const int* __restrict__ nbr,
                      const uint32_t* __restrict__ nbc, const int4* __restrict__ WP,
                      const float4* __restrict__ WN, const float4* __restrict__ acc_prior,
                      float4* __restrict__ acc_keep, Global* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int kb;
  const bool uni = block_one_instance(inst_of, n, &kb);
  bool valid = i < n;
  const int k = valid ? inst_index(inst_of, i) : kb;
  const double dtd = ctrl[k].dt;
  if (dtd == 0.0) valid = false;                 // tank idle for this substep
  float v2 = 0.0f;
  if (valid) {
    const Inst& I = inst[k];
    const float dt = (float)dtd, hdt = 0.5f * dt;
    const float dq = I.dq, inv_h = I.inv_h, dwr = I.dwr_a, rho0 = I.rho0, c0sq = I.c0sq;
    const float c0 = I.c0, kc = kLimiter / c0, qc0 = 0.25f * c0;
    const int px = PER ? I.period[0] : 0, py = PER ? I.period[1] : 0, pz = PER ? I.period[2] : 0;
    const int4 pi = PS[i];
    const float4 vi = VS[i];
    const float dev_i = i2f(pi.w) + hdt * vi.w;       // Eq. verlet-first-half (density)
    const float rho_i = rho0 + dev_i;
    const float pr_i = c0sq * dev_i;                  // Eq. eqeos
    const float2 HDT = f2(hdt), DQ = f2(dq), MAG = f2(-kMagic);
    const float2 VIX = f2(vi.x), VIY = f2(vi.y), VIZ = f2(vi.z);
    float2 sx = f2(0.f), sy = f2(0.f), sz = f2(0.f), nx = f2(0.f), ny = f2(0.f), nz = f2(0.f);
    const uint32_t cnt = nbc[i];
    const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
    const float mi = mass ? 0.0f : I.mass;
    for (int kk = 0; kk < nf; kk += 2) {
      const int ja = nbr[(int64_t)kk * n + i];
      const int jb = kk + 1 < nf ? nbr[(int64_t)(kk + 1) * n + i] : (int)i;   // self pad: zero term
      const int4 pa = PS[ja], pb = PS[jb];
      const float4 va = VS[ja], vb = VS[jb];
      // half-step pair vector r_ij = dq (q_i - q_j) + dt/2 (v_i - v_j)
      const float2 rx = fma2(add2(make_float2(biased_diff<PER>(pi.x, pa.x, px), biased_diff<PER>(pi.x, pb.x, px)), MAG),
                             DQ, mul2(HDT, sub2(VIX, make_float2(va.x, vb.x))));
      const float2 ry = fma2(add2(make_float2(biased_diff<PER>(pi.y, pa.y, py), biased_diff<PER>(pi.y, pb.y, py)), MAG),
                             DQ, mul2(HDT, sub2(VIY, make_float2(va.y, vb.y))));
      float2 rz = f2(0.f);
      if (D == 3)
        rz = fma2(add2(make_float2(biased_diff<PER>(pi.z, pa.z, pz), biased_diff<PER>(pi.z, pb.z, pz)), MAG),
                  DQ, mul2(HDT, sub2(VIZ, make_float2(va.z, vb.z))));
      const Geo2 G = geometry2(rx, ry, rz, inv_h, dwr);
      const float2 dev_j = fma2(HDT, make_float2(va.w, vb.w), make_float2(i2f(pa.w), i2f(pb.w)));
      const float2 rho_j = add2(f2(rho0), dev_j);
      // U_L - U_R = (v_j - v_i).r_ij / |r_ij|
      const float2 vjr = fma2(make_float2(va.x, vb.x), rx, fma2(make_float2(va.y, vb.y), ry,
                              mul2(make_float2(va.z, vb.z), rz)));
      const float2 vir = fma2(VIX, rx, fma2(VIY, ry, mul2(VIZ, rz)));
      const float2 dU = mul2(sub2(vjr, vir), G.inv_r);
      const float2 beta = min2(mul2(f2(kc), max2(dU, 0.0f)), 1.0f);
      // P* = (p_i + p_j)/2 + (c0/4)(rho_i + rho_j) beta (U_L - U_R)
      const float2 pbar = mul2(f2(0.5f * c0sq), add2(f2(dev_i), dev_j));
      const float2 pstar = fma2(mul2(f2(qc0), add2(f2(rho_i), rho_j)), mul2(beta, dU), pbar);
      float2 mj = f2(mi);
      if (mass) mj = make_float2(mass[ja], mass[jb]);
      const float2 f = mul2(mul2(mul2(mj, rcp2(rho_j)), pstar), G.fw);   // V_j P* (dW/dr)/r
      kahan2(sx, nx, f, rx);
      kahan2(sy, ny, f, ry);
      if (D == 3) kahan2(sz, nz, f, rz);
    }
    if (nw) {
      const float g0 = I.g[0], g1 = I.g[1], g2 = I.g[2];
      const float inv_c0sq = 1.0f / c0sq;
      for (int kk = 0; kk < nw; kk += 2) {
        const int wa = nbr[(int64_t)(nf + kk) * n + i];
        const bool has_b = kk + 1 < nw;
        const int wb = has_b ? nbr[(int64_t)(nf + kk + 1) * n + i] : wa;
        const int4 qa = WP[wa], qb = WP[wb];
        const float4 na = WN[wa], nb = WN[wb];
        const float2 rx = fma2(add2(make_float2(biased_diff<PER>(pi.x, qa.x, px), biased_diff<PER>(pi.x, qb.x, px)), MAG),
                               DQ, f2(hdt * vi.x));
        const float2 ry = fma2(add2(make_float2(biased_diff<PER>(pi.y, qa.y, py), biased_diff<PER>(pi.y, qb.y, py)), MAG),
                               DQ, f2(hdt * vi.y));
        float2 rz = f2(0.f);
        if (D == 3)
          rz = fma2(add2(make_float2(biased_diff<PER>(pi.z, qa.z, pz), biased_diff<PER>(pi.z, qb.z, pz)), MAG),
                    DQ, f2(hdt * vi.z));
        const Geo2 G = geometry2(rx, ry, rz, inv_h, dwr);
        // one-sided problem: U_L = -n.v_i, U_R = -U_L, P_R = P_L + rho_i g.(r_w - r_i)
        const float2 UL = mul2(f2(-1.0f), fma2(make_float2(na.x, nb.x), VIX,
                                               fma2(make_float2(na.y, nb.y), VIY, mul2(make_float2(na.z, nb.z), VIZ))));
        const float2 gr = fma2(f2(g0), rx, fma2(f2(g1), ry, mul2(f2(g2), rz)));
        const float2 PR = fma2(f2(-rho_i), gr, f2(pr_i));
        const float2 rhoR = fma2(PR, f2(inv_c0sq), f2(rho0));
        const float2 dU = add2(UL, UL);
        const float2 beta = min2(mul2(f2(kc), max2(dU, 0.0f)), 1.0f);
        const float2 pstar = fma2(mul2(f2(qc0), add2(f2(rho_i), rhoR)), mul2(beta, dU),
                                  mul2(f2(0.5f), add2(f2(pr_i), PR)));
        float2 Vw = make_float2(i2f(qa.w), has_b ? i2f(qb.w) : 0.0f);   // duplicate pad carries no volume
        const float2 f = mul2(mul2(Vw, pstar), G.fw);
        kahan2(sx, nx, f, rx);
        kahan2(sy, ny, f, ry);
        if (D == 3) kahan2(sz, nz, f, rz);
      }
    }
    // dv/dt = acc_prior + g - (2/rho_i) sum V_j P* grad_i W_ij
    const float s = -2.0f / rho_i;
    const float ax = (sx.x + nx.x) + (sx.y + nx.y);
    const float ay = (sy.x + ny.x) + (sy.y + ny.y);
    const float az = (sz.x + nz.x) + (sz.y + nz.y);
    const float4 ap = acc_prior ? acc_prior[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float a0 = ap.x + I.g[0] + s * ax;
    const float a1 = ap.y + I.g[1] + s * ay;
    const float a2 = D == 3 ? ap.z + I.g[2] + s * az : 0.f;
    const float4 vn = make_float4(vi.x + dt * a0, vi.y + dt * a1, vi.z + dt * a2, vi.w);  // verlet-first-mediate
    int qx = pi.x + __float2int_rn(hdt * vi.x * I.inv_dq);                              // verlet-first-half
    int qy = pi.y + __float2int_rn(hdt * vi.y * I.inv_dq);
    int qz = D == 3 ? pi.z + __float2int_rn(hdt * vi.z * I.inv_dq) : 0;
    if (PER) {
      qx = wrap_coord(qx, px);
      qy = wrap_coord(qy, py);
      if (D == 3) qz = wrap_coord(qz, pz);
    }
    PH[i] = make_int4(qx, qy, qz, f2i(dev_i));
    VH[i] = vn;
    if (acc_keep) acc_keep[i] = make_float4(a0, a1, a2, 0.f);
    v2 = vn.x * vn.x + vn.y * vn.y + vn.z * vn.z;
    if (!isfinite(v2)) raise_error(g, ERR_NAN, i);
  }
  reduce_vmax(v2, valid, k, uni, ctrl);
}

// ---------------------------------------------------------------- density relaxation ---
template <int D, bool PER>
__global__ void __launch_bounds__(kBlock, 2)
k_density_relaxation(int64_t n, const int4* __restrict__ PH, const float4* __restrict__ VH,
                     int4* __restrict__ PS, float4* __restrict__ VS,
                     const float* __restrict__ mass, const int* __restrict__ inst_of,
                     const Inst* __restrict__ inst, const Ctrl* __restrict__ ctrl,
                     const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                     const int4* __restrict__ WP, const float4* __restrict__ WN, Global* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = inst_index(inst_of, i);
  const double dtd = ctrl[k].dt;
  if (dtd == 0.0) return;
  const Inst& I = inst[k];
  const float hdt = 0.5f * (float)dtd;
  const float dq = I.dq, inv_h = I.inv_h, dwr = I.dwr_a, rho0 = I.rho0, c0 = I.c0;
  const int px = PER ? I.period[0] : 0, py = PER ? I.period[1] : 0, pz = PER ? I.period[2] : 0;
  const int4 pi = PH[i];
  const float4 vi = VH[i];                            // v^{n+1}
  const float dev_i = i2f(pi.w);
  const float rho_i = rho0 + dev_i;
  const float2 HDT = f2(hdt), DQ = f2(dq), MAG = f2(-kMagic);
  const float2 VIX = f2(vi.x), VIY = f2(vi.y), VIZ = f2(vi.z);
  float2 s = f2(0.f), nc = f2(0.f);
  const uint32_t cnt = nbc[i];
  const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
  const float mi = mass ? 0.0f : I.mass;
  for (int kk = 0; kk < nf; kk += 2) {
    const int ja = nbr[(int64_t)kk * n + i];
    const int jb = kk + 1 < nf ? nbr[(int64_t)(kk + 1) * n + i] : (int)i;
    const int4 pa = PH[ja], pb = PH[jb];
    const float4 va = VH[ja], vb = VH[jb];
    // r_ij^{n+1} = r_ij^{n+1/2} + dt/2 (v_i - v_j)^{n+1}
    const float2 rx = fma2(add2(make_float2(biased_diff<PER>(pi.x, pa.x, px), biased_diff<PER>(pi.x, pb.x, px)), MAG),
                           DQ, mul2(HDT, sub2(VIX, make_float2(va.x, vb.x))));
    const float2 ry = fma2(add2(make_float2(biased_diff<PER>(pi.y, pa.y, py), biased_diff<PER>(pi.y, pb.y, py)), MAG),
                           DQ, mul2(HDT, sub2(VIY, make_float2(va.y, vb.y))));
    float2 rz = f2(0.f);
    if (D == 3)
      rz = fma2(add2(make_float2(biased_diff<PER>(pi.z, pa.z, pz), biased_diff<PER>(pi.z, pb.z, pz)), MAG),
                DQ, mul2(HDT, sub2(VIZ, make_float2(va.z, vb.z))));
    const Geo2 G = geometry2(rx, ry, rz, inv_h, dwr);
    const float2 dev_j = make_float2(i2f(pa.w), i2f(pb.w));
    const float2 rho_j = add2(f2(rho0), dev_j);
    const float2 vjr = fma2(make_float2(va.x, vb.x), rx, fma2(make_float2(va.y, vb.y), ry,
                            mul2(make_float2(va.z, vb.z), rz)));
    const float2 vir = fma2(VIX, rx, fma2(VIY, ry, mul2(VIZ, rz)));
    // U* - U_L = (U_R - U_L)/2 + c0 (dev_i - dev_j)/(rho_i + rho_j)
    const float2 half_dUR = mul2(mul2(sub2(vir, vjr), G.inv_r), f2(0.5f));
    const float2 dUs = fma2(mul2(f2(c0), sub2(f2(dev_i), dev_j)), rcp2(add2(f2(rho_i), rho_j)), half_dUR);
    float2 mj = f2(mi);
    if (mass) mj = make_float2(mass[ja], mass[jb]);
    const float2 dW = mul2(G.fw, G.r);
    kahan2(s, nc, mul2(mul2(mj, rcp2(rho_j)), dUs), dW);
  }
  if (nw) {
    const float g0 = I.g[0], g1 = I.g[1], g2 = I.g[2];
    const float inv_c0sq = 1.0f / I.c0sq, pr_i = I.c0sq * dev_i;
    for (int kk = 0; kk < nw; kk += 2) {
      const int wa = nbr[(int64_t)(nf + kk) * n + i];
      const bool has_b = kk + 1 < nw;
      const int wb = has_b ? nbr[(int64_t)(nf + kk + 1) * n + i] : wa;
      const int4 qa = WP[wa], qb = WP[wb];
      const float4 na = WN[wa], nb = WN[wb];
      const float2 rx = fma2(add2(make_float2(biased_diff<PER>(pi.x, qa.x, px), biased_diff<PER>(pi.x, qb.x, px)), MAG),
                             DQ, f2(hdt * vi.x));
      const float2 ry = fma2(add2(make_float2(biased_diff<PER>(pi.y, qa.y, py), biased_diff<PER>(pi.y, qb.y, py)), MAG),
                             DQ, f2(hdt * vi.y));
      float2 rz = f2(0.f);
      if (D == 3)
        rz = fma2(add2(make_float2(biased_diff<PER>(pi.z, qa.z, pz), biased_diff<PER>(pi.z, qb.z, pz)), MAG),
                  DQ, f2(hdt * vi.z));
      const Geo2 G = geometry2(rx, ry, rz, inv_h, dwr);
      const float2 UL = mul2(f2(-1.0f), fma2(make_float2(na.x, nb.x), VIX,
                                             fma2(make_float2(na.y, nb.y), VIY, mul2(make_float2(na.z, nb.z), VIZ))));
      const float2 gr = fma2(f2(g0), rx, fma2(f2(g1), ry, mul2(f2(g2), rz)));
      const float2 PR = fma2(f2(-rho_i), gr, f2(pr_i));
      const float2 rhoR = fma2(PR, f2(inv_c0sq), f2(rho0));
      // U_R = -U_L: U* = (P_L - P_R)/(2 rho_bar c0) = rho_i g.r_iw / (c0 (rho_i + rho_R))
      const float2 Us = mul2(mul2(f2(rho_i), gr), rcp2(mul2(f2(c0), add2(f2(rho_i), rhoR))));
      const float2 Vw = make_float2(i2f(qa.w), has_b ? i2f(qb.w) : 0.0f);
      kahan2(s, nc, mul2(Vw, sub2(Us, UL)), mul2(G.fw, G.r));
    }
  }
  const float drho = 2.0f * rho_i * ((s.x + nc.x) + (s.y + nc.y));
  const float dev_n = dev_i + hdt * drho;             // Eq. verlet-first-final (density)
  int qx = pi.x + __float2int_rn(hdt * vi.x * I.inv_dq);
  int qy = pi.y + __float2int_rn(hdt * vi.y * I.inv_dq);
  int qz = D == 3 ? pi.z + __float2int_rn(hdt * vi.z * I.inv_dq) : 0;
  if (PER) {
    qx = wrap_coord(qx, px);
    qy = wrap_coord(qy, py);
    if (D == 3) qz = wrap_coord(qz, pz);
  }
  if (!isfinite(dev_n)) raise_error(g, ERR_NAN, i);
  PS[i] = make_int4(qx, qy, qz, f2i(dev_n));
  VS[i] = make_float4(vi.x, vi.y, vi.z, drho);
}

template <typename K2P, typename K2N, typename K3P, typename K3N, typename... A>
void dispatch(const Buffers& b, cudaStream_t s, K2P k2p, K2N k2n, K3P k3p, K3N k3n, A... args) {
  const unsigned grid = grid_for(b.n);
  if (b.dim == 2) {
    if (b.any_periodic) k2p<<<grid, kBlock, 0, s>>>(args...);
    else k2n<<<grid, kBlock, 0, s>>>(args...);
  } else {
    if (b.any_periodic) k3p<<<grid, kBlock, 0, s>>>(args...);
    else k3n<<<grid, kBlock, 0, s>>>(args...);
  }
}

}  // namespace

void launch_pressure_relaxation(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  dispatch(b, s, k_pressure_relaxation<2, true>, k_pressure_relaxation<2, false>,
           k_pressure_relaxation<3, true>, k_pressure_relaxation<3, false>, b.n, (const int4*)b.PS,
           (const float4*)b.VS, b.PH, b.VH, (const float*)b.mass, b.inst_of, (const Inst*)b.inst, b.ctrl,
           (const int*)b.nbr, (const uint32_t*)b.nbc, (const int4*)b.WP, (const float4*)b.WN,
           (const float4*)b.acc_prior, b.acc_keep, b.glob);
  ++*launches;
}

void launch_density_relaxation(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  dispatch(b, s, k_density_relaxation<2, true>, k_density_relaxation<2, false>,
           k_density_relaxation<3, true>, k_density_relaxation<3, false>, b.n, (const int4*)b.PH,
           (const float4*)b.VH, b.PS, b.VS, (const float*)b.mass, b.inst_of, (const Inst*)b.inst,
           (const Ctrl*)b.ctrl, (const int*)b.nbr, (const uint32_t*)b.nbc, (const int4*)b.WP,
           (const float4*)b.WN, b.glob);
  ++*launches;
}

}  // namespace sph
