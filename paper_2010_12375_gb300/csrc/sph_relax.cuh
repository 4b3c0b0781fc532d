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
// One thread per fluid particle walks its frozen neighbour row one quad (four
// slots, one 16-byte load, the next quad already in flight) at a time; the eight
// neighbour records of a quad are gathered together and evaluated as two packed
// pairs in the .x and .y lanes of sm_100 packed FP32 instructions (__ffma2_rn and
// friends), which halves the instruction count of the pair arithmetic. Unused
// slots of the last quad are padded with the particle itself, a pair at zero
// distance whose contribution is exactly zero. Pairs that drifted past 2h get
// t = max(1 - q/2, 0) = 0 and contribute nothing, with no branch. Each lane sums its
// pairs in plain FP32 (one fused multiply-add per term and axis) and the two lanes are
// added at the end: the accumulation error stays near 1e-7 of the sum on every parity
// state, far inside the 1e-5 per-substep bound, and compensated sums cost 8 % of the
// pressure relaxation's time on GB300.
//
// Template switches: TPP threads per particle and BLK threads per block (launch
// variants, each with its own register budget); UNI, a single-tank handle whose constant
// record arrives as the kernel argument; FG, the frozen-geometry reading, where each
// pair's vector r_i - r_j and (dW/dr)/r come from the table written at the configuration
// update instead of from the current positions; TV (pressure relaxation only), the
// transport velocity of Eq. transport, whose background-pressure term moves the mid-point
// position by dt^2/2 a_i.
//
// Launch forms: the per-particle kernels above map thread i of the grid to particle i;
// k_pressure_relaxation_rows / k_density_relaxation_rows (the row-task form, one tank)
// run the same per-particle code in one resident block an SM whose warps take 32-particle
// pieces of the search-cell rows from a queue (see the row-task section below).
#pragma once

#include "sph_kernels.h"

namespace sph {

namespace {

constexpr int kMaxBlock = 512;         // launch variants use 128, 256 or 512 threads

// Resident blocks per SM each launch variant is compiled for (its register budget):
// 896 threads per SM (72 registers) for both relaxation kernels at 128-thread blocks,
// measured fastest on the 8M 3D dam break (more warps in flight hide the neighbour
// gathers better than a larger register budget).
constexpr int pr_min_blocks(int block) { return block == 128 ? 7 : (block == 256 ? 3 : 1); }
constexpr int dr_min_blocks(int block) { return block == 128 ? 7 : (block == 256 ? 3 : 1); }
constexpr float kTinyR2 = 1e-30f;     // keeps rsqrt finite for a pair at zero distance

inline unsigned grid_for(int64_t threads, int block) {
  return (unsigned)((threads + block - 1) / block);
}

// Sum of a value over the TPP consecutive lanes that share a particle, in a fixed
// butterfly order: every lane of the group gets the same, deterministic total.
template <int TPP>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = 1; o < TPP; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void raise_error(Global* g, int bit, long long idx) {
  int old = atomicOr(&g->err, bit);
  if (old == 0) g->bad_index = idx;
}

__device__ __forceinline__ int inst_index(const int* inst_of, int64_t i) {
  return inst_of ? inst_of[i] : 0;
}

// Whether the particles [first, last] of this block (TPP threads each) share one tank.
template <int TPP>
__device__ __forceinline__ bool block_one_instance(const int* inst_of, int64_t n, int* k_out) {
  int64_t first = (int64_t)blockIdx.x * (blockDim.x / TPP);
  int64_t last = min(first + (int64_t)(blockDim.x / TPP), n) - 1;
  if (first > last) last = first;
  int a = inst_index(inst_of, min(first, n - 1)), b = inst_index(inst_of, max(last, (int64_t)0));
  *k_out = a;
  return a == b;
}

__device__ __forceinline__ void reduce_vmax(float v2, bool valid, int k, bool uniform_block, Ctrl* ctrl) {
  __shared__ float red[kMaxBlock / 32];
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

// s += a*b in both lanes (the second argument, the slot a compensated sum would keep, is
// unused: the relaxations sum plainly).
__device__ __forceinline__ void acc2(float2& s, float2&, float2 a, float2 b) { s = fma2(a, b, s); }

// Per-pair kernel factor (dW/dr)/r and |r| from the packed pair vector.
struct Geo2 {
  float2 inv_r, r, fw;
};

__device__ __forceinline__ Geo2 geometry2(float2 rx, float2 ry, float2 rz, float inv_h, float dwr) {
  Geo2 g;
  float2 r2 = fma2(rx, rx, fma2(ry, ry, fma2(rz, rz, f2(kTinyR2))));
  g.inv_r = rsqrt2(r2);
  g.r = mul2(r2, g.inv_r);
  // 1 - q/2 clamped to [0, 1] (0 beyond 2h; r >= 0 keeps it <= 1): one saturating FMA per lane
  float2 t = make_float2(__saturatef(fmaf(g.r.x, -0.5f * inv_h, 1.0f)), __saturatef(fmaf(g.r.y, -0.5f * inv_h, 1.0f)));
  g.fw = mul2(f2(dwr), mul2(mul2(t, t), t));                       // -5 alpha/h^2 (1-q/2)^3
  return g;
}

// The same factors from a stored pair vector and (dW/dr)/r (frozen-geometry reading):
// 1/|r| and |r| come out of the same operations as in geometry2.
__device__ __forceinline__ Geo2 stored_geometry2(float2 rx, float2 ry, float2 rz, float2 fw) {
  Geo2 g;
  float2 r2 = fma2(rx, rx, fma2(ry, ry, fma2(rz, rz, f2(kTinyR2))));
  g.inv_r = rsqrt2(r2);
  g.r = mul2(r2, g.inv_r);
  g.fw = fw;
  return g;
}

// Exactly converted, packed pair vector: dq (q_i - q_j) + add, lanes (a, b).
template <bool PER>
__device__ __forceinline__ float2 pair_axis(int qi, int qa, int qb, int period, float2 DQ, float2 add) {
  return fma2(add2(make_float2(biased_diff<PER>(qi, qa, period), biased_diff<PER>(qi, qb, period)),
                   f2(-kMagic)),
              DQ, add);
}

// Shared per-particle context of the pressure relaxation.
struct PrCtx {
  float hdt, dev_i, rho_i, pr_i;
  int px, py, pz;
  float2 sx, sy, sz, nx, ny, nz;      // per-lane sums (nx, ny, nz stay zero: plain sums)
  float2 bx, by, bz;                  // transport velocity: sum V_j (dW/dr)/r r_ij (plain sums)
};

// Two fluid pairs (a, b) of the pressure relaxation: V_j P* (dW/dr)/r r_ij accumulated.
// FG: the pair vectors and (dW/dr)/r come from the frozen table (ga, gb), else from the
// mid-point positions.
template <int D, bool PER, bool FG = false, bool TV = false>
__device__ __forceinline__ void pr_fluid2(const Inst& I, PrCtx& C, const int4& pi, const float4& vi, const int4& pa,
                                          const int4& pb, const float4& va, const float4& vb, float2 mj,
                                          float2 DQ, float4 ga = float4(), float4 gb = float4()) {
  const float2 HDT = f2(C.hdt), MHDT = f2(-C.hdt);
  // v_j - v_i; hdt (v_i - v_j) = (-hdt)(v_j - v_i) exactly, so one difference serves both
  const float2 dvx = sub2(make_float2(va.x, vb.x), f2(vi.x));
  const float2 dvy = sub2(make_float2(va.y, vb.y), f2(vi.y));
  const float2 dvz = D == 3 ? sub2(make_float2(va.z, vb.z), f2(vi.z)) : f2(0.f);
  float2 rx, ry, rz = f2(0.f);
  Geo2 G;
  if (FG) {
    rx = make_float2(ga.x, gb.x);
    ry = make_float2(ga.y, gb.y);
    if (D == 3) rz = make_float2(ga.z, gb.z);
    G = stored_geometry2(rx, ry, rz, make_float2(ga.w, gb.w));
  } else {
    rx = pair_axis<PER>(pi.x, pa.x, pb.x, C.px, DQ, mul2(MHDT, dvx));
    ry = pair_axis<PER>(pi.y, pa.y, pb.y, C.py, DQ, mul2(MHDT, dvy));
    if (D == 3) rz = pair_axis<PER>(pi.z, pa.z, pb.z, C.pz, DQ, mul2(MHDT, dvz));
    G = geometry2(rx, ry, rz, I.inv_h, I.dwr_a);
  }
  const float2 dev_j = fma2(HDT, make_float2(va.w, vb.w), make_float2(i2f(pa.w), i2f(pb.w)));
  const float2 rho_j = add2(f2(I.rho0), dev_j);
  // U_L - U_R = (v_j - v_i).r_ij / |r_ij|
  const float2 dU = mul2(fma2(dvx, rx, fma2(dvy, ry, mul2(dvz, rz))), G.inv_r);
  const float2 beta = make_float2(__saturatef(I.kc * dU.x), __saturatef(I.kc * dU.y));   // min(kc max(dU, 0), 1)
  // P* = (p_i + p_j)/2 + (c0/4)(rho_i + rho_j) beta (U_L - U_R)
  const float2 pbar = mul2(f2(I.hc0sq), add2(f2(C.dev_i), dev_j));
  const float2 pstar = fma2(mul2(f2(I.qc0), add2(f2(C.rho_i), rho_j)), mul2(beta, dU), pbar);
  const float2 f = mul2(mul2(mul2(mj, rcp2(rho_j)), pstar), G.fw);       // V_j P* (dW/dr)/r
  acc2(C.sx, C.nx, f, rx);
  acc2(C.sy, C.ny, f, ry);
  if (D == 3) acc2(C.sz, C.nz, f, rz);
  if (TV) {                                          // Eq. transport: V_j grad_i W_ij
    const float2 b = mul2(mul2(mj, rcp2(rho_j)), G.fw);
    C.bx = fma2(b, rx, C.bx);
    C.by = fma2(b, ry, C.by);
    if (D == 3) C.bz = fma2(b, rz, C.bz);
  }
}

// Two wall pairs of the pressure relaxation (one-sided problem along the wall normal).
template <int D, bool PER, bool FG = false>
__device__ __forceinline__ void pr_wall2(const Inst& I, PrCtx& C, const int4& pi, const float4& vi,
                                         const int4& qa, const int4& qb, const float4& na,
                                         const float4& nb, float2 Vw, float2 DQ,
                                         float4 ga = float4(), float4 gb = float4()) {
  float2 rx, ry, rz = f2(0.f);
  Geo2 G;
  if (FG) {
    rx = make_float2(ga.x, gb.x);
    ry = make_float2(ga.y, gb.y);
    if (D == 3) rz = make_float2(ga.z, gb.z);
    G = stored_geometry2(rx, ry, rz, make_float2(ga.w, gb.w));
  } else {
    rx = pair_axis<PER>(pi.x, qa.x, qb.x, C.px, DQ, f2(C.hdt * vi.x));
    ry = pair_axis<PER>(pi.y, qa.y, qb.y, C.py, DQ, f2(C.hdt * vi.y));
    if (D == 3) rz = pair_axis<PER>(pi.z, qa.z, qb.z, C.pz, DQ, f2(C.hdt * vi.z));
    G = geometry2(rx, ry, rz, I.inv_h, I.dwr_a);
  }
  // U_L = -n.v_i, U_R = -U_L, P_R = P_L + rho_i g.(r_w - r_i), rho_R from the EoS
  const float2 UL = mul2(f2(-1.0f), fma2(make_float2(na.x, nb.x), f2(vi.x),
                                         fma2(make_float2(na.y, nb.y), f2(vi.y), mul2(make_float2(na.z, nb.z), f2(vi.z)))));
  const float2 gr = fma2(f2(I.g[0]), rx, fma2(f2(I.g[1]), ry, mul2(f2(I.g[2]), rz)));
  const float2 PR = fma2(f2(-C.rho_i), gr, f2(C.pr_i));
  const float2 rhoR = fma2(PR, f2(I.inv_c0sq), f2(I.rho0));
  const float2 dU = add2(UL, UL);
  const float2 beta = make_float2(__saturatef(I.kc * dU.x), __saturatef(I.kc * dU.y));   // min(kc max(dU, 0), 1)
  const float2 pstar = fma2(mul2(f2(I.qc0), add2(f2(C.rho_i), rhoR)), mul2(beta, dU),
                            mul2(f2(0.5f), add2(f2(C.pr_i), PR)));
  const float2 f = mul2(mul2(Vw, pstar), G.fw);
  acc2(C.sx, C.nx, f, rx);
  acc2(C.sy, C.ny, f, ry);
  if (D == 3) acc2(C.sz, C.nz, f, rz);
}

// ---------------------------------------------------------------- pressure relaxation --
// TPP threads share one particle: lane `sub` takes quads sub, sub + TPP, ... of its row,
// and the lanes' compensated sums are combined in a fixed order. TPP = 1 is one thread per
// particle; 2 and 4 trade per-thread work for more threads in flight.
// FG: pair geometry from the frozen table geo ([slot][n]) instead of the positions.
// TV: transport velocity (Eq. transport): the mid-point position written for the density
// relaxation also takes dt^2/2 a_i, a_i = -(2 p0 / rho_i) sum_j V_j grad_i W_ij over the
// fluid pairs (one thread per particle only).
// One particle of the pressure relaxation, lane `sub` of the TPP lanes that share it (all
// lanes take part in the group shuffles, valid or not). Returns |v^{n+1}|^2 on the lane
// that wrote the particle (*writer), else 0. The array pointers carry the caller's
// aliasing qualifiers: the per-launch kernels pass __restrict__ ones, the persistent
// loop plain ones (its phases read what other blocks wrote in the previous phase).
template <int D, bool PER, int TPP, bool FG, bool TV, typename PI, typename PF>
__device__ __forceinline__ float pr_particle(const Inst& I, int64_t i, int sub, bool valid, double dtd,
                                             const float4* __restrict__ geo, int64_t n, PI PS, PF VS,
                                             int4* PH, float4* VH, const float* __restrict__ mass,
                                             const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                                             const int4* __restrict__ WP, const float4* __restrict__ WN,
                                             const float4* __restrict__ acc_prior, float4* __restrict__ acc_keep,
                                             Global* g, bool* writer_out) {
  float v2 = 0.0f;
  static_assert(!TV || (TPP == 1 && !FG), "transport velocity: one thread per particle, recomputed geometry");
  PrCtx C;
  C.sx = C.sy = C.sz = C.nx = C.ny = C.nz = f2(0.f);
  C.bx = C.by = C.bz = f2(0.f);
  const float dt = (float)dtd;
  int4 pi = make_int4(0, 0, 0, 0);
  float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    C.hdt = 0.5f * dt;
    C.px = PER ? I.period[0] : 0;
    C.py = PER ? I.period[1] : 0;
    C.pz = PER ? I.period[2] : 0;
    pi = PS[i];
    vi = VS[i];
    C.dev_i = i2f(pi.w) + C.hdt * vi.w;               // Eq. verlet-first-half (density)
    C.rho_i = I.rho0 + C.dev_i;
    C.pr_i = I.c0sq * C.dev_i;                        // Eq. eqeos
    const float2 DQ = f2(I.dq);
    const uint32_t cnt = nbc[i];
    const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
    const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
    const int nq = (nf + 3) >> 2;
    int4 cur = sub < nq ? nb4[(int64_t)sub * n + i] : make_int4(0, 0, 0, 0);
    for (int q = sub; q < nq; q += TPP) {
      int4 nxt = cur;
      if (q + TPP < nq) nxt = nb4[(int64_t)(q + TPP) * n + i];  // next quad in flight
      const int s = q << 2;
      const int j0 = cur.x;
      const int j1 = s + 1 < nf ? cur.y : (int)i;                // self pads: zero terms
      const int j2 = s + 2 < nf ? cur.z : (int)i;
      const int j3 = s + 3 < nf ? cur.w : (int)i;
      int4 p0, p1, p2, p3;
      float4 g0 = float4(), g1 = float4(), g2 = float4(), g3 = float4();
      if (FG) {                                  // the frozen table holds the geometry: only dev_j here
        const int* __restrict__ dw = reinterpret_cast<const int*>(PS) + 3;
        p0 = make_int4(0, 0, 0, dw[4 * (int64_t)j0]);
        p1 = make_int4(0, 0, 0, dw[4 * (int64_t)j1]);
        p2 = make_int4(0, 0, 0, dw[4 * (int64_t)j2]);
        p3 = make_int4(0, 0, 0, dw[4 * (int64_t)j3]);
        const float4* __restrict__ gq = geo + (int64_t)s * n + i;
        g0 = gq[0];
        g1 = gq[n];
        g2 = gq[2 * n];
        g3 = gq[3 * n];
      } else {
        p0 = PS[j0];
        p1 = PS[j1];
        p2 = PS[j2];
        p3 = PS[j3];
      }
      const float4 v0 = VS[j0], v1 = VS[j1], v2v = VS[j2], v3 = VS[j3];
      float2 m01 = f2(I.mass), m23 = f2(I.mass);
      if (mass) {
        m01 = make_float2(mass[j0], mass[j1]);
        m23 = make_float2(mass[j2], mass[j3]);
      }
      pr_fluid2<D, PER, FG, TV>(I, C, pi, vi, p0, p1, v0, v1, m01, DQ, g0, g1);
      pr_fluid2<D, PER, FG, TV>(I, C, pi, vi, p2, p3, v2v, v3, m23, DQ, g2, g3);
      cur = nxt;
    }
    if (nw) {
      const int q0 = wall_slot0(nf) >> 2, nwq = (nw + 3) >> 2;
      for (int q = sub; q < nwq; q += TPP) {
        const int4 c = nb4[(int64_t)(q0 + q) * n + i];
        const int s = q << 2;
        const int w1 = s + 1 < nw ? c.y : c.x, w2 = s + 2 < nw ? c.z : c.x, w3 = s + 3 < nw ? c.w : c.x;
        const int4 a0 = WP[c.x], a1 = WP[w1], a2 = WP[w2], a3 = WP[w3];
        const float4 n0 = WN[c.x], n1 = WN[w1], n2 = WN[w2], n3 = WN[w3];
        const float2 V01 = make_float2(i2f(a0.w), s + 1 < nw ? i2f(a1.w) : 0.0f);   // pads carry no volume
        const float2 V23 = make_float2(s + 2 < nw ? i2f(a2.w) : 0.0f, s + 3 < nw ? i2f(a3.w) : 0.0f);
        float4 g0 = float4(), g1 = float4(), g2 = float4(), g3 = float4();
        if (FG) {
          const float4* __restrict__ gq = geo + (int64_t)((q0 + q) << 2) * n + i;
          g0 = gq[0];
          g1 = gq[n];
          g2 = gq[2 * n];
          g3 = gq[3 * n];
        }
        pr_wall2<D, PER, FG>(I, C, pi, vi, a0, a1, n0, n1, V01, DQ, g0, g1);
        pr_wall2<D, PER, FG>(I, C, pi, vi, a2, a3, n2, n3, V23, DQ, g2, g3);
      }
    }
  }
  // per-lane compensated sums, then the group total (all lanes take part in the shuffles)
  float ax = (C.sx.x + C.nx.x) + (C.sx.y + C.nx.y);
  float ay = (C.sy.x + C.ny.x) + (C.sy.y + C.ny.y);
  float az = (C.sz.x + C.nz.x) + (C.sz.y + C.nz.y);
  if (TPP > 1) {
    ax = group_sum<TPP>(ax);
    ay = group_sum<TPP>(ay);
    if (D == 3) az = group_sum<TPP>(az);
  }
  const bool writer = valid && sub == 0;
  if (writer) {
    // dv/dt = acc_prior + g - (2/rho_i) sum V_j P* grad_i W_ij
    const float sc = -2.0f / C.rho_i;
    const float4 ap = acc_prior ? acc_prior[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float a0 = ap.x + I.g[0] + sc * ax;
    const float a1 = ap.y + I.g[1] + sc * ay;
    const float a2 = D == 3 ? ap.z + I.g[2] + sc * az : 0.f;
    const float4 vn = make_float4(vi.x + dt * a0, vi.y + dt * a1, vi.z + dt * a2, vi.w);  // verlet-first-mediate
    const float hdt = C.hdt;
    float ux = vi.x, uy = vi.y, uz = vi.z;                   // dt/2 times this moves r to n+1/2
    if (TV) {                                                // + dt^2/2 a_i: dt/2 (v + dt a_i)
      const float tv = -2.0f * I.p_tv / C.rho_i * dt;
      ux += tv * (C.bx.x + C.bx.y);
      uy += tv * (C.by.x + C.by.y);
      uz += tv * (C.bz.x + C.bz.y);
    }
    int qx = pi.x + __float2int_rn(hdt * ux * I.inv_dq);                                // verlet-first-half
    int qy = pi.y + __float2int_rn(hdt * uy * I.inv_dq);
    int qz = D == 3 ? pi.z + __float2int_rn(hdt * uz * I.inv_dq) : 0;
    if (PER) {
      qx = wrap_coord(qx, C.px);
      qy = wrap_coord(qy, C.py);
      if (D == 3) qz = wrap_coord(qz, C.pz);
    }
    PH[i] = make_int4(qx, qy, qz, f2i(C.dev_i));
    VH[i] = vn;
    if (acc_keep) acc_keep[i] = make_float4(a0, a1, a2, 0.f);
    v2 = vn.x * vn.x + vn.y * vn.y + vn.z * vn.z;
    if (!isfinite(v2)) raise_error(g, ERR_NAN, i);
  }
  *writer_out = writer;
  return v2;
}

template <int D, bool PER, int TPP, int BLK, bool UNI, bool FG, bool TV = false>
__global__ void __launch_bounds__(BLK, pr_min_blocks(BLK))
k_pressure_relaxation(const Inst Ip, const float4* __restrict__ geo, int64_t n, const int4* __restrict__ PS,
                      const float4* __restrict__ VS,
                      int4* __restrict__ PH, float4* __restrict__ VH,
                      const float* __restrict__ mass, const int* __restrict__ inst_of,
                      const Inst* __restrict__ inst, Ctrl* ctrl, const int* __restrict__ nbr,
                      const uint32_t* __restrict__ nbc, const int4* __restrict__ WP,
                      const float4* __restrict__ WN, const float4* __restrict__ acc_prior,
                      float4* __restrict__ acc_keep, Global* g) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
  const int sub = TPP > 1 ? (int)(threadIdx.x % TPP) : 0;
  int kb;
  const bool uni = block_one_instance<TPP>(inst_of, n, &kb);
  bool valid = i < n;
  const int k = valid ? inst_index(inst_of, i) : kb;
  const double dtd = ctrl[k].dt;
  if (dtd == 0.0) valid = false;                 // tank idle for this substep
  const Inst& I = UNI ? Ip : inst[k];        // one tank: constants straight from the argument
  bool writer;
  const float v2 = pr_particle<D, PER, TPP, FG, TV, const int4* __restrict__, const float4* __restrict__>(
      I, i, sub, valid, dtd, geo, n, PS, VS, PH, VH, mass, nbr, nbc, WP, WN, acc_prior, acc_keep, g, &writer);
  reduce_vmax(v2, writer, k, uni, ctrl);
}

// ---------------------------------------------------------------- density relaxation ---
struct DrCtx {
  float hdt, dev_i, rho_i;
  int px, py, pz;
  float2 s, nc;
};

template <int D, bool PER, bool FG = false>
__device__ __forceinline__ void dr_fluid2(const Inst& I, DrCtx& C, const int4& pi, const float4& vi, const int4& pa,
                                          const int4& pb, const float4& va, const float4& vb, float2 mj,
                                          float2 DQ, float4 ga = float4(), float4 gb = float4()) {
  const float2 HDT = f2(C.hdt);
  float2 rx, ry, rz = f2(0.f);
  Geo2 G;
  if (FG) {
    rx = make_float2(ga.x, gb.x);
    ry = make_float2(ga.y, gb.y);
    if (D == 3) rz = make_float2(ga.z, gb.z);
    G = stored_geometry2(rx, ry, rz, make_float2(ga.w, gb.w));
  } else {
    // r_ij^{n+1} = r_ij^{n+1/2} + dt/2 (v_i - v_j)^{n+1}
    rx = pair_axis<PER>(pi.x, pa.x, pb.x, C.px, DQ, mul2(HDT, sub2(f2(vi.x), make_float2(va.x, vb.x))));
    ry = pair_axis<PER>(pi.y, pa.y, pb.y, C.py, DQ, mul2(HDT, sub2(f2(vi.y), make_float2(va.y, vb.y))));
    if (D == 3) rz = pair_axis<PER>(pi.z, pa.z, pb.z, C.pz, DQ, mul2(HDT, sub2(f2(vi.z), make_float2(va.z, vb.z))));
    G = geometry2(rx, ry, rz, I.inv_h, I.dwr_a);
  }
  const float2 dev_j = make_float2(i2f(pa.w), i2f(pb.w));
  const float2 rho_j = add2(f2(I.rho0), dev_j);
  // (U_R - U_L)/2 = (v_i - v_j).r_ij / (2 |r_ij|)
  const float2 dvx = sub2(f2(vi.x), make_float2(va.x, vb.x));
  const float2 dvy = sub2(f2(vi.y), make_float2(va.y, vb.y));
  const float2 dvz = sub2(f2(vi.z), make_float2(va.z, vb.z));
  const float2 half_dUR = mul2(fma2(dvx, rx, fma2(dvy, ry, mul2(dvz, rz))), mul2(G.inv_r, f2(0.5f)));
  // U* - U_L = (U_R - U_L)/2 + c0 (dev_i - dev_j)/(rho_i + rho_j)
  const float2 dUs = fma2(mul2(f2(I.c0), sub2(f2(C.dev_i), dev_j)), rcp2(add2(f2(C.rho_i), rho_j)), half_dUR);
  acc2(C.s, C.nc, mul2(mul2(mj, rcp2(rho_j)), dUs), mul2(G.fw, G.r));
}

template <int D, bool PER, bool FG = false>
__device__ __forceinline__ void dr_wall2(const Inst& I, DrCtx& C, const int4& pi, const float4& vi,
                                         const int4& qa, const int4& qb, const float4& na,
                                         const float4& nb, float2 Vw, float2 DQ, float pr_i,
                                         float4 ga = float4(), float4 gb = float4()) {
  float2 rx, ry, rz = f2(0.f);
  Geo2 G;
  if (FG) {
    rx = make_float2(ga.x, gb.x);
    ry = make_float2(ga.y, gb.y);
    if (D == 3) rz = make_float2(ga.z, gb.z);
    G = stored_geometry2(rx, ry, rz, make_float2(ga.w, gb.w));
  } else {
    rx = pair_axis<PER>(pi.x, qa.x, qb.x, C.px, DQ, f2(C.hdt * vi.x));
    ry = pair_axis<PER>(pi.y, qa.y, qb.y, C.py, DQ, f2(C.hdt * vi.y));
    if (D == 3) rz = pair_axis<PER>(pi.z, qa.z, qb.z, C.pz, DQ, f2(C.hdt * vi.z));
    G = geometry2(rx, ry, rz, I.inv_h, I.dwr_a);
  }
  const float2 UL = mul2(f2(-1.0f), fma2(make_float2(na.x, nb.x), f2(vi.x),
                                         fma2(make_float2(na.y, nb.y), f2(vi.y), mul2(make_float2(na.z, nb.z), f2(vi.z)))));
  const float2 gr = fma2(f2(I.g[0]), rx, fma2(f2(I.g[1]), ry, mul2(f2(I.g[2]), rz)));
  const float2 PR = fma2(f2(-C.rho_i), gr, f2(pr_i));
  const float2 rhoR = fma2(PR, f2(I.inv_c0sq), f2(I.rho0));
  // U_R = -U_L: U* = (P_L - P_R)/(2 rho_bar c0) = rho_i g.r_iw / (c0 (rho_i + rho_R))
  const float2 Us = mul2(mul2(f2(C.rho_i), gr), rcp2(mul2(f2(I.c0), add2(f2(C.rho_i), rhoR))));
  acc2(C.s, C.nc, mul2(Vw, sub2(Us, UL)), mul2(G.fw, G.r));
}

// One particle of the density relaxation, lane `sub` of TPP (pointer qualifiers as for
// pr_particle).
template <int D, bool PER, int TPP, bool FG, typename PI, typename PF>
__device__ __forceinline__ void dr_particle(const Inst& I, int64_t i, int sub, bool valid, double dtd,
                                            const float4* __restrict__ geo, int64_t n, PI PH, PF VH,
                                            int4* PS, float4* VS, const float* __restrict__ mass,
                                            const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                                            const int4* __restrict__ WP, const float4* __restrict__ WN, Global* g) {
  DrCtx C;
  C.s = C.nc = f2(0.f);
  int4 pi = make_int4(0, 0, 0, 0);
  float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
  C.hdt = 0.5f * (float)dtd;
  if (valid) {
    C.px = PER ? I.period[0] : 0;
    C.py = PER ? I.period[1] : 0;
    C.pz = PER ? I.period[2] : 0;
    pi = PH[i];
    vi = VH[i];                                       // v^{n+1}
    C.dev_i = i2f(pi.w);
    C.rho_i = I.rho0 + C.dev_i;
    const float2 DQ = f2(I.dq);
    const uint32_t cnt = nbc[i];
    const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
    const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
    const int nq = (nf + 3) >> 2;
    int4 cur = sub < nq ? nb4[(int64_t)sub * n + i] : make_int4(0, 0, 0, 0);
    for (int q = sub; q < nq; q += TPP) {
      int4 nxt = cur;
      if (q + TPP < nq) nxt = nb4[(int64_t)(q + TPP) * n + i];
      const int s = q << 2;
      const int j0 = cur.x;
      const int j1 = s + 1 < nf ? cur.y : (int)i;
      const int j2 = s + 2 < nf ? cur.z : (int)i;
      const int j3 = s + 3 < nf ? cur.w : (int)i;
      int4 p0, p1, p2, p3;
      float4 g0 = float4(), g1 = float4(), g2 = float4(), g3 = float4();
      if (FG) {                                  // the frozen table holds the geometry: only dev_j here
        const int* __restrict__ dw = reinterpret_cast<const int*>(PH) + 3;
        p0 = make_int4(0, 0, 0, dw[4 * (int64_t)j0]);
        p1 = make_int4(0, 0, 0, dw[4 * (int64_t)j1]);
        p2 = make_int4(0, 0, 0, dw[4 * (int64_t)j2]);
        p3 = make_int4(0, 0, 0, dw[4 * (int64_t)j3]);
        const float4* __restrict__ gq = geo + (int64_t)s * n + i;
        g0 = gq[0];
        g1 = gq[n];
        g2 = gq[2 * n];
        g3 = gq[3 * n];
      } else {
        p0 = PH[j0];
        p1 = PH[j1];
        p2 = PH[j2];
        p3 = PH[j3];
      }
      const float4 v0 = VH[j0], v1 = VH[j1], v2 = VH[j2], v3 = VH[j3];
      float2 m01 = f2(I.mass), m23 = f2(I.mass);
      if (mass) {
        m01 = make_float2(mass[j0], mass[j1]);
        m23 = make_float2(mass[j2], mass[j3]);
      }
      dr_fluid2<D, PER, FG>(I, C, pi, vi, p0, p1, v0, v1, m01, DQ, g0, g1);
      dr_fluid2<D, PER, FG>(I, C, pi, vi, p2, p3, v2, v3, m23, DQ, g2, g3);
      cur = nxt;
    }
    if (nw) {
      const float pr_i = I.c0sq * C.dev_i;
      const int q0 = wall_slot0(nf) >> 2, nwq = (nw + 3) >> 2;
      for (int q = sub; q < nwq; q += TPP) {
        const int4 c = nb4[(int64_t)(q0 + q) * n + i];
        const int s = q << 2;
        const int w1 = s + 1 < nw ? c.y : c.x, w2 = s + 2 < nw ? c.z : c.x, w3 = s + 3 < nw ? c.w : c.x;
        const int4 a0 = WP[c.x], a1 = WP[w1], a2 = WP[w2], a3 = WP[w3];
        const float4 n0 = WN[c.x], n1 = WN[w1], n2 = WN[w2], n3 = WN[w3];
        const float2 V01 = make_float2(i2f(a0.w), s + 1 < nw ? i2f(a1.w) : 0.0f);
        const float2 V23 = make_float2(s + 2 < nw ? i2f(a2.w) : 0.0f, s + 3 < nw ? i2f(a3.w) : 0.0f);
        float4 g0 = float4(), g1 = float4(), g2 = float4(), g3 = float4();
        if (FG) {
          const float4* __restrict__ gq = geo + (int64_t)((q0 + q) << 2) * n + i;
          g0 = gq[0];
          g1 = gq[n];
          g2 = gq[2 * n];
          g3 = gq[3 * n];
        }
        dr_wall2<D, PER, FG>(I, C, pi, vi, a0, a1, n0, n1, V01, DQ, pr_i, g0, g1);
        dr_wall2<D, PER, FG>(I, C, pi, vi, a2, a3, n2, n3, V23, DQ, pr_i, g2, g3);
      }
    }
  }
  float sum = (C.s.x + C.nc.x) + (C.s.y + C.nc.y);
  if (TPP > 1) sum = group_sum<TPP>(sum);
  if (!valid || sub != 0) return;
  const float drho = 2.0f * C.rho_i * sum;
  const float dev_n = C.dev_i + C.hdt * drho;         // Eq. verlet-first-final (density)
  const float hdt = C.hdt;
  int qx = pi.x + __float2int_rn(hdt * vi.x * I.inv_dq);
  int qy = pi.y + __float2int_rn(hdt * vi.y * I.inv_dq);
  int qz = D == 3 ? pi.z + __float2int_rn(hdt * vi.z * I.inv_dq) : 0;
  if (PER) {
    qx = wrap_coord(qx, C.px);
    qy = wrap_coord(qy, C.py);
    if (D == 3) qz = wrap_coord(qz, C.pz);
  }
  if (!isfinite(dev_n)) raise_error(g, ERR_NAN, i);
  PS[i] = make_int4(qx, qy, qz, f2i(dev_n));
  VS[i] = make_float4(vi.x, vi.y, vi.z, drho);
}

template <int D, bool PER, int TPP, int BLK, bool UNI, bool FG>
__global__ void __launch_bounds__(BLK, dr_min_blocks(BLK))
k_density_relaxation(const Inst Ip, const float4* __restrict__ geo, int64_t n, const int4* __restrict__ PH,
                     const float4* __restrict__ VH,
                     int4* __restrict__ PS, float4* __restrict__ VS,
                     const float* __restrict__ mass, const int* __restrict__ inst_of,
                     const Inst* __restrict__ inst, const Ctrl* __restrict__ ctrl,
                     const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                     const int4* __restrict__ WP, const float4* __restrict__ WN, Global* g) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
  const int sub = TPP > 1 ? (int)(threadIdx.x % TPP) : 0;
  if (TPP == 1 && i >= n) return;                     // no group shuffles to take part in
  bool valid = i < n;
  const int k = valid ? inst_index(inst_of, i) : 0;
  const double dtd = ctrl[k].dt;
  if (TPP == 1 && dtd == 0.0) return;
  if (dtd == 0.0) valid = false;
  const Inst& I = UNI ? Ip : inst[k];        // one tank: constants straight from the argument
  dr_particle<D, PER, TPP, FG, const int4* __restrict__, const float4* __restrict__>(
      I, i, sub, valid, dtd, geo, n, PH, VH, PS, VS, mass, nbr, nbc, WP, WN, g);
}

// ---------------------------------------------------------------- row-task form ---
// One resident block of kRowWarps warps an SM, one thread per particle. Each warp takes
// the next piece (32 consecutive particles of one search-cell row, `row_task`) from its
// block's queue: block b works through the runs of kRowWarps consecutive pieces numbered
// b, b + gridDim.x, b + 2 gridDim.x, ..., so the blocks move through the cell order side by
// side (the rows in flight share their neighbours in L1 and L2) and a warp that finishes
// early takes the next piece instead of waiting for the rest of its block. The particle
// arithmetic is that of the one-thread-per-particle kernels: results equal theirs bit for bit.
__device__ __forceinline__ bool next_row_piece(int* queue, int lane, long long pieces, long long* t_out) {
  int q = 0;
  if (lane == 0) q = atomicAdd(queue, 1);
  q = __shfl_sync(0xffffffffu, q, 0);
  const long long t = ((long long)blockIdx.x + (long long)gridDim.x * (q / kRowWarps)) * kRowWarps + q % kRowWarps;
  *t_out = t;
  return t < pieces;
}

template <int D, bool PER, bool TV>
__global__ void __launch_bounds__(kRowBlock, 1)
k_pressure_relaxation_rows(const Inst I, int64_t n, const int4* __restrict__ PS, const float4* __restrict__ VS,
                           int4* __restrict__ PH, float4* __restrict__ VH, const float* __restrict__ mass,
                           Ctrl* ctrl, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                           const int4* __restrict__ WP, const float4* __restrict__ WN,
                           const float4* __restrict__ acc_prior, float4* __restrict__ acc_keep, Global* g,
                           const int2* __restrict__ row_task, const uint32_t* __restrict__ row_total,
                           int64_t row_task_cap) {
  __shared__ int queue;
  __shared__ float red[kRowWarps];
  if (threadIdx.x == 0) queue = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long pieces = min((long long)*row_total, (long long)row_task_cap);
  const double dtd = ctrl[0].dt;
  float m = 0.0f;
  long long t;
  if (dtd != 0.0) {                              // 0: the tank is idle for this substep
    while (next_row_piece(&queue, lane, pieces, &t)) {
      const int2 piece = row_task[t];
      const bool valid = lane < piece.y;
      bool writer;
      const float v2 = pr_particle<D, PER, 1, false, TV, const int4* __restrict__, const float4* __restrict__>(
          I, valid ? (int64_t)piece.x + lane : 0, 0, valid, dtd, nullptr, n, PS, VS, PH, VH, mass, nbr, nbc,
          WP, WN, acc_prior, acc_keep, g, &writer);
      if (writer) m = fmaxf(m, v2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < kRowWarps ? red[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(&ctrl[0].vmax2, __float_as_uint(m));
  }
}

template <int D, bool PER>
__global__ void __launch_bounds__(kRowBlock, 1)
k_density_relaxation_rows(const Inst I, int64_t n, const int4* __restrict__ PH, const float4* __restrict__ VH,
                          int4* __restrict__ PS, float4* __restrict__ VS, const float* __restrict__ mass,
                          const Ctrl* __restrict__ ctrl, const int* __restrict__ nbr,
                          const uint32_t* __restrict__ nbc, const int4* __restrict__ WP,
                          const float4* __restrict__ WN, Global* g, const int2* __restrict__ row_task,
                          const uint32_t* __restrict__ row_total, int64_t row_task_cap) {
  __shared__ int queue;
  if (threadIdx.x == 0) queue = 0;
  __syncthreads();
  const double dtd = ctrl[0].dt;
  if (dtd == 0.0) return;
  const int lane = threadIdx.x & 31;
  const long long pieces = min((long long)*row_total, (long long)row_task_cap);
  long long t;
  while (next_row_piece(&queue, lane, pieces, &t)) {
    const int2 piece = row_task[t];
    const bool valid = lane < piece.y;
    dr_particle<D, PER, 1, false, const int4* __restrict__, const float4* __restrict__>(
        I, valid ? (int64_t)piece.x + lane : 0, 0, valid, dtd, nullptr, n, PH, VH, PS, VS, mass, nbr, nbc,
        WP, WN, g);
  }
}

// Launch variants: (threads per particle, block size) per kernel, indexed by kTpp / kBlk.
template <int D, bool PER>
void launch_pr(int tpp, int block, const Buffers& b, cudaStream_t s) {
  const unsigned grid = grid_for(b.n * tpp, block);
#define SPH_PR_ARGS b.n, (const int4*)b.PS, (const float4*)b.VS, b.PH, b.VH, (const float*)b.mass, \
    b.inst_of, (const Inst*)b.inst, b.ctrl, (const int*)b.nbr, (const uint32_t*)b.nbc,                 \
    (const int4*)b.WP, (const float4*)b.WN, (const float4*)b.acc_prior, b.acc_keep, b.glob
  // one instantiation per (threads per particle, block) pair, each with its own bounds
#define SPH_PR(T, B) (b.n_inst == 1                                                                 \
      ? k_pressure_relaxation<D, PER, T, B, true, false><<<grid, B, 0, s>>>(b.inst0, nullptr, SPH_PR_ARGS) \
      : k_pressure_relaxation<D, PER, T, B, false, false><<<grid, B, 0, s>>>(b.inst0, nullptr, SPH_PR_ARGS))
  if (b.geo) {               // frozen geometry: one variant, one thread per particle
    const unsigned g1 = grid_for(b.n, 128);
    if (b.n_inst == 1) k_pressure_relaxation<D, PER, 1, 128, true, true><<<g1, 128, 0, s>>>(b.inst0, b.geo, SPH_PR_ARGS);
    else k_pressure_relaxation<D, PER, 1, 128, false, true><<<g1, 128, 0, s>>>(b.inst0, b.geo, SPH_PR_ARGS);
    return;
  }
  if (row_form(block)) {     // row-task form (one tank; the caller has built the pieces)
#define SPH_PR_ROWS(TV) k_pressure_relaxation_rows<D, PER, TV><<<b.n_sm, kRowBlock, 0, s>>>(                     \
      b.inst0, b.n, (const int4*)b.PS, (const float4*)b.VS, b.PH, b.VH, (const float*)b.mass, b.ctrl,          \
      (const int*)b.nbr, (const uint32_t*)b.nbc, (const int4*)b.WP, (const float4*)b.WN,                        \
      (const float4*)b.acc_prior, b.acc_keep, b.glob, b.row_task, b.row_off + b.n_rows, b.row_task_cap)
    if (b.any_transport) SPH_PR_ROWS(true);
    else SPH_PR_ROWS(false);
#undef SPH_PR_ROWS
    return;
  }
  if (b.any_transport) {     // transport velocity: one thread per particle, the configured block
    const unsigned g1 = grid_for(b.n, block);
#define SPH_PR_TV(B) (b.n_inst == 1                                                                \
      ? k_pressure_relaxation<D, PER, 1, B, true, false, true><<<g1, B, 0, s>>>(b.inst0, nullptr, SPH_PR_ARGS) \
      : k_pressure_relaxation<D, PER, 1, B, false, false, true><<<g1, B, 0, s>>>(b.inst0, nullptr, SPH_PR_ARGS))
    if (block == 512) SPH_PR_TV(512);
    else if (block == 256) SPH_PR_TV(256);
    else SPH_PR_TV(128);
#undef SPH_PR_TV
    return;
  }
#define SPH_PR_T(T) (block == 512 ? SPH_PR(T, 512) : block == 256 ? SPH_PR(T, 256) : SPH_PR(T, 128))
  if (tpp == 4) SPH_PR_T(4);
  else if (tpp == 2) SPH_PR_T(2);
  else SPH_PR_T(1);
#undef SPH_PR_T
#undef SPH_PR
#undef SPH_PR_ARGS
}

template <int D, bool PER>
void launch_dr(int tpp, int block, const Buffers& b, cudaStream_t s) {
  const unsigned grid = grid_for(b.n * tpp, block);
#define SPH_DR_ARGS b.n, (const int4*)b.PH, (const float4*)b.VH, b.PS, b.VS, (const float*)b.mass, \
    b.inst_of, (const Inst*)b.inst, (const Ctrl*)b.ctrl, (const int*)b.nbr, (const uint32_t*)b.nbc,   \
    (const int4*)b.WP, (const float4*)b.WN, b.glob
#define SPH_DR(T, B) (b.n_inst == 1                                                                 \
      ? k_density_relaxation<D, PER, T, B, true, false><<<grid, B, 0, s>>>(b.inst0, nullptr, SPH_DR_ARGS) \
      : k_density_relaxation<D, PER, T, B, false, false><<<grid, B, 0, s>>>(b.inst0, nullptr, SPH_DR_ARGS))
  if (b.geo) {
    const unsigned g1 = grid_for(b.n, 128);
    if (b.n_inst == 1) k_density_relaxation<D, PER, 1, 128, true, true><<<g1, 128, 0, s>>>(b.inst0, b.geo, SPH_DR_ARGS);
    else k_density_relaxation<D, PER, 1, 128, false, true><<<g1, 128, 0, s>>>(b.inst0, b.geo, SPH_DR_ARGS);
    return;
  }
  if (row_form(block)) {     // row-task form (one tank; the caller has built the pieces)
    k_density_relaxation_rows<D, PER><<<b.n_sm, kRowBlock, 0, s>>>(
        b.inst0, b.n, (const int4*)b.PH, (const float4*)b.VH, b.PS, b.VS, (const float*)b.mass,
        (const Ctrl*)b.ctrl, (const int*)b.nbr, (const uint32_t*)b.nbc, (const int4*)b.WP, (const float4*)b.WN,
        b.glob, b.row_task, b.row_off + b.n_rows, b.row_task_cap);
    return;
  }
#define SPH_DR_T(T) (block == 512 ? SPH_DR(T, 512) : block == 256 ? SPH_DR(T, 256) : SPH_DR(T, 128))
  if (tpp == 4) SPH_DR_T(4);
  else if (tpp == 2) SPH_DR_T(2);
  else SPH_DR_T(1);
#undef SPH_DR_T
#undef SPH_DR
#undef SPH_DR_ARGS
}

}  // namespace

}  // namespace sph
