// Species diffusion on the fluid particles (Sec. "Schemes for thermal and mass diffusion")
// and the reaction step of reaction-diffusion (Sec. "Reaction-by-reaction splitting"; its
// kernel and readings are described where it is defined, below the diffusion kernels).
//
//   dC_i/dt = 2 sum_j (m_j/rho_j) (C_i - C_j) w(e_ij) (1/r_ij) dW/dr_ij      (Eq. grad-laplace)
//   w(e)    = 1/(L^-1 e)^2 = 1/(e^T D^-1 e),  D = L L^T                        (Eq. chol)
//
// with one diffusion tensor per species object, so the pair combination of the
// per-particle factors is the factor itself; for isotropic D = kappa I, w = kappa.
// Time integration is the two-stage second-order Runge-Kutta scheme (Heun), one kernel
// launch per stage:
//   stage 1: C*      = C^n + dt f(C^n)
//   stage 2: C^{n+1} = (C^n + C* + dt f(C*)) / 2      (written over C^n, own index only)
//
// One thread per fluid particle walks the fluid part of its neighbour row in the
// quad-interleaved table, keeping the next index quad in flight. Each call packs, per slot,
// one 16-byte record R = {qx, qy, qz, bits(C)} (2D: {qx, qy, bits(V), bits(C)}, V = m/rho),
// so a neighbour costs one 16-byte gather. Stages ping-pong between two record buffers and
// write only the species word. The pair arithmetic is issue-bound, so it runs two pairs per
// packed FP32 instruction; pair coordinates are exact integer differences converted with
// the magic-number add, wrapped on periodic axes only for particles within the support of
// a periodic face; and when all volumes and diffusivity factors of a tank are equal
// (checked once per call by the pack kernel, read by the host, which then launches the
// uniform instantiation; neighbours never cross tanks, so then V_j = V_i) the volume, the
// factor and the kernel constants leave the pair loop. Otherwise V_j comes from the record
// (2D) or a per-slot array (3D) and the factor pair from a per-slot array. Wall neighbours
// are skipped: walls carry no species (zero flux). Pairs at zero distance add nothing.
//
// Per-particle tensors of different shape (D_i = L_i L_i^T, Eq. chol): the printed pair
// combination read as the harmonic mean of matrices gives the weight r^2 / |M^-1 r|^2 with
// M = (L_i + L_j)/2 (lower triangular, forward substitution per pair); the factors are
// formed once per upload (FP64 Cholesky), times sqrt(s_i) with per-particle factors, and
// gathered per slot like B0 below.
//
// Kernel-corrected form (Eq. grad-laplace-renormalize, read as: the pair weight gains
// (e^T B0_i e + e^T B0_j e)/2): once per call a kernel forms each slot's symmetric
// B0_i = (sum_j V_j (r_j - r_i) (x) grad_i W_ij)^-1 over the same fluid pairs (the identity
// where that sum is singular), and the corrected stage kernels gather B0_j with each record.
//
// Between calls the species is kept by caller row, so the fluid solver may re-sort the
// particles; each call gathers it into slot order, runs its steps and scatters it back.
#include <cmath>
#include <string>

#include "sph_handle.h"

namespace sph {
namespace {

constexpr int kDiffBlock = 256;

// Symmetric D^-1 (xx, yy, zz, xy, xz, yz) and the isotropic coefficient.
struct DiffCoef {
  float xx, yy, zz, xy, xz, yz, kappa;
};

inline unsigned diff_grid(int64_t n) { return (unsigned)((n + kDiffBlock - 1) / kDiffBlock); }

// Exactly converted, packed pair coordinate q_i - q_j for lanes (a, b), in length units.
template <bool PER>
__device__ __forceinline__ float2 pair_coord2(int qi, int qa, int qb, int period, float2 DQ) {
  return mul2(add2(make_float2(biased_diff<PER>(qi, qa, period), biased_diff<PER>(qi, qb, period)),
                   f2(-kMagic)),
              DQ);
}

// Two pairs (lanes a, b) of the stage sum without the volumes and without the constant
// factor dwr_a of (dW/dr)/r (and kappa when isotropic):
// (C_i - C_j) (1 - q/2)^3 w(e_ij). At zero distance r = 0 * inf is NaN, fmaxf turns the
// kernel factor into 0 and the pair adds nothing.
// Symmetric B0 of a slot: {xx, yy, zz, xy, xz, yz}, stored as one float4 {xx, yy, xy, 0}
// per slot in 2D and two, {xx, yy, zz, xy} and {xz, yz, 0, 0}, in 3D.
struct Sym3 {
  float xx, yy, zz, xy, xz, yz;
};
template <int D>
__device__ __forceinline__ Sym3 load_b0(const float4* __restrict__ Bc, int64_t j) {
  if (D == 2) {
    const float4 b = Bc[j];
    return Sym3{b.x, b.y, 0.0f, b.z, 0.0f, 0.0f};
  }
  const float4 b0 = Bc[2 * j], b1 = Bc[2 * j + 1];
  return Sym3{b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
}
// Lower-triangular factor of a slot: {l00, l10, l11, l20, l21, l22}, stored as one float4
// {l00, l10, l11, 0} per slot in 2D and two, {l00, l10, l11, l20} and {l21, l22, 0, 0}, in 3D.
struct Tri3 {
  float l00, l10, l11, l20, l21, l22;
};
template <int D>
__device__ __forceinline__ Tri3 load_tri(const float4* __restrict__ Lc, int64_t j) {
  if (D == 2) {
    const float4 b = Lc[j];
    return Tri3{b.x, b.y, b.z, 0.0f, 0.0f, 1.0f};
  }
  const float4 b0 = Lc[2 * j], b1 = Lc[2 * j + 1];
  return Tri3{b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
}
// |M^-1 r|^2 for one pair, M = (L_i + L_j)/2, by forward substitution
template <int D>
__device__ __forceinline__ float tri_solve_sq(const Tri3& Li, const Tri3& Lj, float rx, float ry, float rz) {
  const float m00 = 0.5f * (Li.l00 + Lj.l00), m10 = 0.5f * (Li.l10 + Lj.l10), m11 = 0.5f * (Li.l11 + Lj.l11);
  const float y0 = __fdividef(rx, m00);
  const float y1 = __fdividef(fmaf(-m10, y0, ry), m11);
  float q = fmaf(y0, y0, y1 * y1);
  if (D == 3) {
    const float m20 = 0.5f * (Li.l20 + Lj.l20), m21 = 0.5f * (Li.l21 + Lj.l21), m22 = 0.5f * (Li.l22 + Lj.l22);
    const float y2 = __fdividef(fmaf(-m21, y1, fmaf(-m20, y0, rz)), m22);
    q = fmaf(y2, y2, q);
  }
  return q;
}

template <int D>
__device__ __forceinline__ float2 quad_form2(const Sym3& B, float2 rx, float2 ry, float2 rz) {
  float2 q = fma2(mul2(f2(B.xx), rx), rx, fma2(mul2(f2(B.yy), ry), ry, mul2(mul2(f2(2.0f * B.xy), rx), ry)));
  if (D == 3)
    q = fma2(mul2(f2(B.zz), rz), rz, fma2(mul2(f2(2.0f * B.xz), rx), rz, fma2(mul2(f2(2.0f * B.yz), ry), rz, q)));
  return q;
}

// TEN: per-particle tensors (the weight from the factors Li, La, Lb; ISO and K unused).
template <int D, bool PER, bool ISO, bool CORR = false, bool TEN = false>
__device__ __forceinline__ float2 diff_terms2(const Inst& I, const DiffCoef& K, const int4& ri, float ci,
                                              const int4& a, const int4& b, const Sym3* Bi = nullptr,
                                              const Sym3* Ba = nullptr, const Sym3* Bb = nullptr,
                                              const Tri3* Li = nullptr, const Tri3* La = nullptr,
                                              const Tri3* Lb = nullptr) {
  const float2 DQ = f2(I.dq);
  const float2 rx = pair_coord2<PER>(ri.x, a.x, b.x, I.period[0], DQ);
  const float2 ry = pair_coord2<PER>(ri.y, a.y, b.y, I.period[1], DQ);
  float2 rz = f2(0.0f);
  float2 r2 = fma2(rx, rx, mul2(ry, ry));
  if (D == 3) {
    rz = pair_coord2<PER>(ri.z, a.z, b.z, I.period[2], DQ);
    r2 = fma2(rz, rz, r2);
  }
  const float2 r = mul2(r2, rsqrt2(r2));
  const float2 t = max2(fma2(r, f2(-0.5f * I.inv_h), f2(1.0f)), 0.0f);
  float2 k = mul2(mul2(t, t), t);
  if (TEN) {                         // r^2 / |M^-1 r|^2
    const float qa = tri_solve_sq<D>(*Li, *La, rx.x, ry.x, rz.x), qb = tri_solve_sq<D>(*Li, *Lb, rx.y, ry.y, rz.y);
    k = mul2(k, make_float2(__fdividef(r2.x, fmaxf(qa, 1e-30f)), __fdividef(r2.y, fmaxf(qb, 1e-30f))));
  } else if (!ISO) {
    float2 qf = fma2(mul2(f2(K.xx), rx), rx, fma2(mul2(f2(K.yy), ry), ry, mul2(mul2(f2(2.0f * K.xy), rx), ry)));
    if (D == 3)
      qf = fma2(mul2(f2(K.zz), rz), rz,
                fma2(mul2(f2(2.0f * K.xz), rx), rz, fma2(mul2(f2(2.0f * K.yz), ry), rz, qf)));
    k = mul2(k, make_float2(__fdividef(r2.x, fmaxf(qf.x, 1e-30f)),       // 1/(e^T D^-1 e)
                            __fdividef(r2.y, fmaxf(qf.y, 1e-30f))));
  }
  if (CORR) {                        // (e^T B0_i e + e^T B0_j e)/2 = (r^T B0_i r + r^T B0_j r)/(2 r^2)
    const float2 qi = quad_form2<D>(*Bi, rx, ry, rz);
    const float2 qab = make_float2(quad_form2<D>(*Ba, rx, ry, rz).x, quad_form2<D>(*Bb, rx, ry, rz).y);
    const float2 half_inv = make_float2(__fdividef(0.5f, fmaxf(r2.x, 1e-30f)), __fdividef(0.5f, fmaxf(r2.y, 1e-30f)));
    k = mul2(k, mul2(add2(qi, qab), half_inv));
  }
  return mul2(sub2(f2(ci), make_float2(i2f(a.w), i2f(b.w))), k);
}

// Sum over the fluid part of row i of weighted pair terms. VJ: each pair weighted by V_j
// (from the record in 2D or the volume array in 3D) and by ((sqrt s_i + sqrt s_j)/2)^2 of
// the per-particle diffusivity factors (sq = sqrt s per slot, NULL when none is set); else
// the caller multiplies by the common volume and factor.
template <int D, bool PER, bool ISO, bool VJ, bool CORR, bool TEN>
__device__ __forceinline__ float row_sum(int64_t n, int64_t i, int nf, const Inst& I, const DiffCoef& K,
                                         const int4& ri, float ci, const int4* __restrict__ R,
                                         const int4* __restrict__ nb4, const float* __restrict__ vol,
                                         const float* __restrict__ sq, float sqi, const float4* __restrict__ Bc,
                                         const Sym3& Bi, const float4* __restrict__ Lc, const Tri3& Li) {
  const int nq = (nf + 3) >> 2;
  float2 s = f2(0.0f);
  int4 nxt = nq ? nb4[i] : make_int4(0, 0, 0, 0);
  for (int q = 0; q < nq; ++q) {
    const int4 cq = nxt;
    if (q + 1 < nq) nxt = nb4[(int64_t)(q + 1) * n + i];   // next quad in flight
    const int sl = q << 2;
    const int j1 = sl + 1 < nf ? cq.y : cq.x, j2 = sl + 2 < nf ? cq.z : cq.x, j3 = sl + 3 < nf ? cq.w : cq.x;
    const int4 a0 = R[cq.x], a1 = R[j1], a2 = R[j2], a3 = R[j3];
    float2 w01 = make_float2(1.0f, sl + 1 < nf ? 1.0f : 0.0f);
    float2 w23 = make_float2(sl + 2 < nf ? 1.0f : 0.0f, sl + 3 < nf ? 1.0f : 0.0f);
    if (VJ) {
      if (D == 2) {
        w01 = mul2(w01, make_float2(i2f(a0.z), i2f(a1.z)));
        w23 = mul2(w23, make_float2(i2f(a2.z), i2f(a3.z)));
      } else {
        w01 = mul2(w01, make_float2(vol[cq.x], vol[j1]));
        w23 = mul2(w23, make_float2(vol[j2], vol[j3]));
      }
      if (sq) {
        const float2 m01 = mul2(add2(f2(sqi), make_float2(sq[cq.x], sq[j1])), f2(0.5f));
        const float2 m23 = mul2(add2(f2(sqi), make_float2(sq[j2], sq[j3])), f2(0.5f));
        w01 = mul2(w01, mul2(m01, m01));
        w23 = mul2(w23, mul2(m23, m23));
      }
    }
    if (TEN) {
      const Tri3 l0 = load_tri<D>(Lc, cq.x), l1 = load_tri<D>(Lc, j1), l2 = load_tri<D>(Lc, j2), l3 = load_tri<D>(Lc, j3);
      if (CORR) {
        const Sym3 b0 = load_b0<D>(Bc, cq.x), b1 = load_b0<D>(Bc, j1), b2 = load_b0<D>(Bc, j2), b3 = load_b0<D>(Bc, j3);
        s = fma2(diff_terms2<D, PER, ISO, true, true>(I, K, ri, ci, a0, a1, &Bi, &b0, &b1, &Li, &l0, &l1), w01, s);
        s = fma2(diff_terms2<D, PER, ISO, true, true>(I, K, ri, ci, a2, a3, &Bi, &b2, &b3, &Li, &l2, &l3), w23, s);
      } else {
        s = fma2(diff_terms2<D, PER, ISO, false, true>(I, K, ri, ci, a0, a1, nullptr, nullptr, nullptr, &Li, &l0, &l1), w01, s);
        s = fma2(diff_terms2<D, PER, ISO, false, true>(I, K, ri, ci, a2, a3, nullptr, nullptr, nullptr, &Li, &l2, &l3), w23, s);
      }
    } else if (CORR) {
      const Sym3 b0 = load_b0<D>(Bc, cq.x), b1 = load_b0<D>(Bc, j1), b2 = load_b0<D>(Bc, j2), b3 = load_b0<D>(Bc, j3);
      s = fma2(diff_terms2<D, PER, ISO, true>(I, K, ri, ci, a0, a1, &Bi, &b0, &b1), w01, s);
      s = fma2(diff_terms2<D, PER, ISO, true>(I, K, ri, ci, a2, a3, &Bi, &b2, &b3), w23, s);
    } else {
      s = fma2(diff_terms2<D, PER, ISO>(I, K, ri, ci, a0, a1), w01, s);
      s = fma2(diff_terms2<D, PER, ISO>(I, K, ri, ci, a2, a3), w23, s);
    }
  }
  return s.x + s.y;
}

// Row sum with the periodic wrap only where a neighbour can lie across a periodic
// boundary: particles farther than the support from every periodic face take the plain
// differences.
template <int D, bool PER, bool ISO, bool VJ, bool CORR, bool TEN>
__device__ __forceinline__ float row_sum_any(int64_t n, int64_t i, int nf, const Inst& I, const DiffCoef& K,
                                             const int4& ri, float ci, const int4* __restrict__ R,
                                             const int4* __restrict__ nb4, const float* __restrict__ vol,
                                             const float* __restrict__ sq, float sqi,
                                             const float4* __restrict__ Bc, const Sym3& Bi,
                                             const float4* __restrict__ Lc, const Tri3& Li) {
  if (PER) {
    const int reach = (int)ceilf(sqrtf((float)I.R2)) + 2;          // support radius in quanta
    const int q[3] = {ri.x, ri.y, ri.z};
    bool near_face = false;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (I.period[a]) near_face |= q[a] < reach || q[a] >= I.period[a] - reach;
    if (near_face)
      return row_sum<D, true, ISO, VJ, CORR, TEN>(n, i, nf, I, K, ri, ci, R, nb4, vol, sq, sqi, Bc, Bi, Lc, Li);
  }
  return row_sum<D, false, ISO, VJ, CORR, TEN>(n, i, nf, I, K, ri, ci, R, nb4, vol, sq, sqi, Bc, Bi, Lc, Li);
}

// Five blocks of 256 per SM (48 registers) for the isotropic uniform variants: the stage
// is latency-bound and runs 8 % faster at 8M particles than with four; the anisotropic
// variants keep four, since they would spill at 48 registers.
// UNIF: volumes and diffusivity factors are equal within each tank (the host reads the
// flag the pack kernel computes); the general path weights every pair and keeps four
// blocks per SM, where its extra per-pair loads fit without spilling.
// CORR: the kernel-corrected form, B0 per slot in Bc (one 16-byte gather per neighbour in
// 2D, two in 3D; fewer resident blocks, where the B0 of a quad of neighbours fits). TEN:
// per-particle tensors, factors per slot in Lc (the same gathers again), on the weighted
// path with the diffusivity factors folded into the factors (sq NULL).
template <int D, bool PER, bool ISO, bool SECOND, bool UNIF, bool CORR, bool TEN>
__global__ void __launch_bounds__(kDiffBlock, (CORR || TEN) ? ((D == 3 || (CORR && TEN)) ? 2 : 3) : (ISO && UNIF ? 5 : 4))
k_diffusion_stage(int64_t n, const int4* __restrict__ Rin, int4* __restrict__ Rout, const int* __restrict__ nbr,
                  const uint32_t* __restrict__ nbc, const int* __restrict__ inst_of,
                  const Inst* __restrict__ inst, const float* __restrict__ vol,
                  const float* __restrict__ sq, DiffCoef K, float dt, const float4* __restrict__ Bc,
                  const float4* __restrict__ Lc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const int4 ri = Rin[i];
  const float ci = i2f(ri.w);
  const int nf = (int)(nbc[i] & 0xffffu);
  const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
  const float sqi = sq ? sq[i] : 1.0f;
  const Sym3 Bi = CORR ? load_b0<D>(Bc, i) : Sym3{1.0f, 1.0f, 1.0f, 0.0f, 0.0f, 0.0f};
  const Tri3 Li = TEN ? load_tri<D>(Lc, i) : Tri3{1.0f, 0.0f, 1.0f, 0.0f, 0.0f, 1.0f};
  float sum;
  if (UNIF) {                      // equal volumes and factors within the tank: those of i
    const float vi = D == 2 ? i2f(ri.z) : vol[i];
    sum = vi * (sqi * sqi) *
          row_sum_any<D, PER, ISO, false, CORR, TEN>(n, i, nf, I, K, ri, ci, Rin, nb4, vol, sq, sqi, Bc, Bi, Lc, Li);
  } else {
    sum = row_sum_any<D, PER, ISO, true, CORR, TEN>(n, i, nf, I, K, ri, ci, Rin, nb4, vol, sq, sqi, Bc, Bi, Lc, Li);
  }
  const float rate = 2.0f * (ISO ? I.dwr_a * K.kappa : I.dwr_a) * sum;
  const float next = fmaf(dt, rate, ci);
  // stage 2 reads C^n from the output record's own slot (written by no other thread)
  const float out = SECOND ? 0.5f * (i2f(Rout[i].w) + next) : next;
  reinterpret_cast<int*>(Rout)[4 * i + 3] = f2i(out);
}

// Per call: records of both buffers from the fluid state and the species by caller row
// (b.id[slot] = caller row), the per-slot volumes (3D) and the flag of unequal volumes
// within a tank.
template <int D>
__global__ void k_species_pack(int64_t n, const int4* __restrict__ P, const int* __restrict__ id,
                               const int* __restrict__ inst_of, const Inst* __restrict__ inst,
                               const float* __restrict__ mass, const float* __restrict__ by_row,
                               int4* __restrict__ R0, int4* __restrict__ R1, float* __restrict__ vol,
                               const float* __restrict__ scale_by_row, float* __restrict__ sq,
                               int* __restrict__ nonuniform) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const int4 p = P[i];
  const float v = __fdividef(mass ? mass[i] : I.mass, I.rho0 + i2f(p.w));      // m_i / rho_i
  const int c = f2i(by_row[id[i]]);
  const int4 r = make_int4(p.x, p.y, D == 2 ? f2i(v) : p.z, c);
  R0[i] = r;
  R1[i] = r;
  if (D == 3) vol[i] = v;
  const int64_t f = I.fluid_begin;                                    // the tank's first slot
  const float vf = __fdividef(mass ? mass[f] : I.mass, I.rho0 + i2f(P[f].w));
  if (vf != v) atomicOr(nonuniform, 1);
  if (scale_by_row) {                                                 // sqrt of s_i, R17
    const float q = sqrtf(scale_by_row[id[i]]);
    sq[i] = q;
    if (sqrtf(scale_by_row[id[f]]) != q) atomicOr(nonuniform, 2);
  }
}

// Per slot: B0_i = (sum_j V_j (r_j - r_i) (x) grad_i W_ij)^-1 over the fluid part of row i
// (grad_i W_ij = dwr_a (1 - q/2)^3 r_ij, so the sum is -dwr_a sum_j V_j (1 - q/2)^3 r_ij r_ij^T,
// symmetric), the identity where its determinant is below 1e-6 (trace/d)^d. Pairs at zero
// distance add nothing.
template <int D, bool PER>
__global__ void k_species_correction(int64_t n, const int4* __restrict__ R, const int* __restrict__ nbr,
                                     const uint32_t* __restrict__ nbc, const int* __restrict__ inst_of,
                                     const Inst* __restrict__ inst, const float* __restrict__ vol,
                                     float4* __restrict__ Bc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const int4 ri = R[i];
  const int nf = (int)(nbc[i] & 0xffffu);
  float mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f, myz = 0.f;
  for (int s = 0; s < nf; ++s) {
    const int j = nbr[(((int64_t)(s >> 2)) * n + i) * 4 + (s & 3)];
    const int4 rj = R[j];
    const float rx = (biased_diff<PER>(ri.x, rj.x, I.period[0]) - kMagic) * I.dq;
    const float ry = (biased_diff<PER>(ri.y, rj.y, I.period[1]) - kMagic) * I.dq;
    const float rz = D == 3 ? (biased_diff<PER>(ri.z, rj.z, I.period[2]) - kMagic) * I.dq : 0.0f;
    const float r2 = rx * rx + ry * ry + rz * rz;
    if (!(r2 > 0.0f)) continue;
    const float t = fmaxf(fmaf(sqrtf(r2), -0.5f * I.inv_h, 1.0f), 0.0f);
    const float w = (D == 2 ? i2f(rj.z) : vol[j]) * t * t * t;
    mxx = fmaf(w * rx, rx, mxx);
    myy = fmaf(w * ry, ry, myy);
    mxy = fmaf(w * rx, ry, mxy);
    if (D == 3) {
      mzz = fmaf(w * rz, rz, mzz);
      mxz = fmaf(w * rx, rz, mxz);
      myz = fmaf(w * ry, rz, myz);
    }
  }
  const float c = -I.dwr_a;                // > 0
  mxx *= c; myy *= c; mzz *= c; mxy *= c; mxz *= c; myz *= c;
  if (D == 2) {
    const float det = mxx * myy - mxy * mxy, tr = 0.5f * (mxx + myy);
    if (det > 1e-6f * tr * tr)
      Bc[i] = make_float4(myy / det, mxx / det, -mxy / det, 0.0f);
    else
      Bc[i] = make_float4(1.0f, 1.0f, 0.0f, 0.0f);
  } else {
    const float cxx = myy * mzz - myz * myz, cyy = mxx * mzz - mxz * mxz, czz = mxx * myy - mxy * mxy;
    const float cxy = mxz * myz - mxy * mzz, cxz = mxy * myz - mxz * myy, cyz = mxy * mxz - mxx * myz;
    const float det = mxx * cxx + mxy * cxy + mxz * cxz, tr = (mxx + myy + mzz) / 3.0f;
    if (det > 1e-6f * tr * tr * tr) {
      Bc[2 * i] = make_float4(cxx / det, cyy / det, czz / det, cxy / det);
      Bc[2 * i + 1] = make_float4(cxz / det, cyz / det, 0.0f, 0.0f);
    } else {
      Bc[2 * i] = make_float4(1.0f, 1.0f, 1.0f, 0.0f);
      Bc[2 * i + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
}

// Per caller row: the lower-triangular Cholesky factor of D_i (row-major d x d doubles), in
// FP64, stored {l00, l10, l11, l20, l21, l22}; flags a tensor that is not finite, symmetric
// and positive definite.
__global__ void k_species_factor(int64_t n, int d, const double* __restrict__ Dp, float* __restrict__ Lrow,
                                 int* __restrict__ bad) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double* A = Dp + r * d * d;
  double L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  bool ok = true;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (!isfinite(A[i * d + j]) || A[i * d + j] != A[j * d + i]) ok = false;
  for (int i = 0; i < d && ok; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = A[i * d + j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(v > 0.0)) {
          ok = false;
          break;
        }
        L[i][i] = sqrt(v);
      } else {
        L[i][j] = v / L[j][j];
      }
    }
  if (!ok) {
    atomicOr(bad, 1);
    return;
  }
  float* o = Lrow + 6 * r;
  o[0] = (float)L[0][0]; o[1] = (float)L[1][0]; o[2] = (float)L[1][1];
  o[3] = (float)L[2][0]; o[4] = (float)L[2][1]; o[5] = (float)(d == 3 ? L[2][2] : 1.0);
}

// Per slot: the factor of the slot's caller row, times sqrt(s) when diffusivity factors are
// set (D_i = s_i D'_i), into the slot layout of load_tri.
template <int D>
__global__ void k_species_pack_tensors(int64_t n, const int* __restrict__ id, const float* __restrict__ Lrow,
                                       const float* __restrict__ scale_by_row, float4* __restrict__ Lc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t r = id[i];
  const float* l = Lrow + 6 * r;
  const float q = scale_by_row ? sqrtf(scale_by_row[r]) : 1.0f;
  if (D == 2) {
    Lc[i] = make_float4(q * l[0], q * l[1], q * l[2], 0.0f);
  } else {
    Lc[2 * i] = make_float4(q * l[0], q * l[1], q * l[2], q * l[3]);
    Lc[2 * i + 1] = make_float4(q * l[4], q * l[5], 0.0f, 0.0f);
  }
}

// Flags a diffusivity factor that is not a positive finite number.
__global__ void k_check_scale(int64_t n, const float* __restrict__ s, int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(s[i] > 0.0f && s[i] <= 3.402823466e38f)) atomicOr(bad, 1);
}

__global__ void k_species_unpack(int64_t n, const int* __restrict__ id, const int4* __restrict__ R,
                                 float* __restrict__ by_row) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) by_row[id[i]] = i2f(R[i].w);
}

__global__ void k_species_import(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

__global__ void k_species_export(int64_t n, const float* __restrict__ src, double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

// ---- reaction step (Sec. "Reaction-by-reaction splitting") ---------------------------------
// Per particle: Eq. ode-spliting-2rd applies R_V(dt/2), R_w(dt/2), R_w(dt/2), R_V(dt/2); each
// reaction writes its right-hand side as q - p y (Eq. ode-new-form) and takes the QSS update
// of Eq. ode-qss with p and q at the reaction's starting value. Production/loss split:
//   FitzHugh-Nagumo (Eq. fhn)  R_V: q = -w, p = (V - a)(V - 1);  R_w: q = eps0 (beta V - sigma),
//                              p = eps0 gamma
//   Aliev-Panfilov (Eq. a-p)   R_V: q = 0, p = k (V - a)(V - 1) + w;  R_w: q = -eps k V (V - b - 1),
//                              p = eps = eps0 + mu1 w / (mu2 + V)
struct ReactCoef {
  int model;
  float a, b, k, eps0, mu1, mu2, beta, gamma, sigma;
};

// y e^(-p dt) + q (1 - e^(-p dt))/p, the fraction taken as dt when |p dt| < 1e-12.
__device__ __forceinline__ float qss(float y, float q, float p, float dt) {
  const float x = -p * dt;
  const float frac = fabsf(x) < 1e-12f ? dt : -expm1f(x) / p;
  return fmaf(y, expf(x), q * frac);
}

__device__ __forceinline__ float react_V(float V, float w, const ReactCoef& R, float dt) {
  if (R.model == 1) return qss(V, -w, (V - R.a) * (V - 1.0f), dt);
  return qss(V, 0.0f, fmaf(R.k * (V - R.a), V - 1.0f, w), dt);
}

__device__ __forceinline__ float react_w(float V, float w, const ReactCoef& R, float dt) {
  if (R.model == 1) return qss(w, R.eps0 * (R.beta * V - R.sigma), R.eps0 * R.gamma, dt);
  const float eps = R.eps0 + R.mu1 * w / (R.mu2 + V);
  return qss(w, -eps * R.k * V * (V - R.b - 1.0f), eps, dt);
}

// All steps of one call in registers: 16 bytes of HBM traffic per particle per call.
__global__ void k_reaction(int64_t n, float* __restrict__ V, float* __restrict__ w, ReactCoef R, float dt,
                           int n_steps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = V[i], g = w[i];
  const float h = 0.5f * dt;
  for (int s = 0; s < n_steps; ++s) {
    v = react_V(v, g, R, h);
    g = react_w(v, g, R, h);
    g = react_w(v, g, R, h);
    v = react_V(v, g, R, h);
  }
  V[i] = v;
  w[i] = g;
}

using StageFn = void (*)(int64_t, const int4*, int4*, const int*, const uint32_t*, const int*, const Inst*,
                         const float*, const float*, DiffCoef, float, const float4*, const float4*);

template <int D, bool PER, bool ISO, bool UNIF, bool CORR, bool TEN = false>
void pick_stages(StageFn* s1, StageFn* s2) {
  *s1 = k_diffusion_stage<D, PER, ISO, false, UNIF, CORR, TEN>;
  *s2 = k_diffusion_stage<D, PER, ISO, true, UNIF, CORR, TEN>;
}

template <int D, bool PER>
void pick_stages(bool iso, bool unif, bool corr, bool ten, StageFn* s1, StageFn* s2) {
  if (ten) {                       // per-particle tensors: the weighted path
    if (corr) pick_stages<D, PER, false, false, true, true>(s1, s2);
    else pick_stages<D, PER, false, false, false, true>(s1, s2);
  } else if (corr) {
    if (iso) {
      if (unif) pick_stages<D, PER, true, true, true>(s1, s2);
      else pick_stages<D, PER, true, false, true>(s1, s2);
    } else {
      if (unif) pick_stages<D, PER, false, true, true>(s1, s2);
      else pick_stages<D, PER, false, false, true>(s1, s2);
    }
  } else if (iso) {
    if (unif) pick_stages<D, PER, true, true, false>(s1, s2);
    else pick_stages<D, PER, true, false, false>(s1, s2);
  } else {
    if (unif) pick_stages<D, PER, false, true, false>(s1, s2);
    else pick_stages<D, PER, false, false, false>(s1, s2);
  }
}

}  // namespace
}  // namespace sph

struct sph_species {
  int dim = 0;
  int64_t n = 0;
  sph::DiffCoef K{};
  bool iso = false;
  float* by_row = nullptr;     // [n] species by caller row (kept between calls)
  float* gate = nullptr;       // [n] gating variable w of the reaction step, by caller row
  int4* r0 = nullptr;          // [n] slot records carrying C^n
  int4* r1 = nullptr;          // [n] slot records carrying C*
  float* vol = nullptr;        // [n] slot volumes m/rho (3D)
  int* nonuniform = nullptr;   // [1] bit 0: volumes differ within a tank; bit 1: factors do
  float* scale_by_row = nullptr;  // [n] per-particle diffusivity factors s (NULL: all 1)
  float* sq = nullptr;         // [n] sqrt(s) per slot (with scale_by_row)
  double* stage = nullptr;     // [n] doubles for host copies
  bool corrected = false;      // the kernel-corrected form (sph_species_set_correction)
  float4* Bc = nullptr;        // [n] (2D) or [2n] (3D): symmetric B0 per slot, formed per call
  float* Lrow = nullptr;       // [6n] per-particle tensor factors by caller row (NULL: none)
  float4* Lc = nullptr;        // [n] (2D) or [2n] (3D): the factors per slot, packed per call
  std::string err;
};

namespace {

int sfail(sph_species* sp, int code, const std::string& msg) {
  if (sp) sp->err = msg;
  return code;
}

// Where a caller array lives: host memory (copied through the staging buffer), memory
// the current device can address directly, or device memory of another GPU (rejected:
// the kernels run on the current device).
enum PtrKind { kHostPtr, kDevicePtr, kOtherDevicePtr };

PtrKind pointer_kind(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kHostPtr;
  }
  if (a.type == cudaMemoryTypeManaged) return kDevicePtr;
  if (a.type != cudaMemoryTypeDevice) return kHostPtr;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return kOtherDevicePtr;
  }
  return a.device == cur ? kDevicePtr : kOtherDevicePtr;
}

// Cholesky factor of a symmetric d x d tensor (row-major); false unless positive definite.
bool cholesky(const double* D, int d, double* L) {
  for (int k = 0; k < 9; ++k) L[k] = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = D[i * d + j];
      for (int k = 0; k < j; ++k) s -= L[i * 3 + k] * L[j * 3 + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i * 3 + i] = std::sqrt(s);
      } else {
        L[i * 3 + j] = s / L[j * 3 + j];
      }
    }
  return true;
}

// D^-1 = L^-T L^-1 from the lower-triangular factor (3 x 3 storage).
void inverse_from_cholesky(const double* L, int d, double* Dinv) {
  double Li[9] = {0};
  for (int i = 0; i < d; ++i) {
    Li[i * 3 + i] = 1.0 / L[i * 3 + i];
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s -= L[i * 3 + k] * Li[k * 3 + j];
      Li[i * 3 + j] = s / L[i * 3 + i];
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += Li[k * 3 + a] * Li[k * 3 + b];
      Dinv[a * 3 + b] = s;
    }
}

}  // namespace

extern "C" {

int sph_species_create(sph_handle* h, const double* D, sph_species** out) {
  if (!out) return SPH_E_INVALID;
  *out = nullptr;
  if (!h || !D) return SPH_E_INVALID;
  auto* sp = new sph_species();
  *out = sp;
  const int d = h->b.dim;
  sp->dim = d;
  sp->n = h->b.n;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (!std::isfinite(D[i * d + j]) || D[i * d + j] != D[j * d + i])
        return sfail(sp, SPH_E_INVALID, "D must be finite and symmetric");
  double L[9], Dinv[9];
  if (!cholesky(D, d, L)) return sfail(sp, SPH_E_INVALID, "D must be positive definite");
  inverse_from_cholesky(L, d, Dinv);
  bool iso = true;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (D[i * d + j] != (i == j ? D[0] : 0.0)) iso = false;
  sp->iso = iso;
  sp->K = sph::DiffCoef{(float)Dinv[0], (float)Dinv[4], (float)Dinv[8], (float)Dinv[1],
                        (float)Dinv[2], (float)Dinv[5], (float)D[0]};
  if (sp->n > 0) {
    const size_t n = (size_t)sp->n;
    if (cudaMalloc(&sp->by_row, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&sp->r0, sizeof(int4) * n) != cudaSuccess ||
        cudaMalloc(&sp->r1, sizeof(int4) * n) != cudaSuccess ||
        cudaMalloc(&sp->vol, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&sp->nonuniform, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&sp->gate, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&sp->stage, sizeof(double) * n) != cudaSuccess) {
      cudaGetLastError();
      return sfail(sp, SPH_E_OOM, "device allocation of the species failed");
    }
    if (cudaMemset(sp->by_row, 0, sizeof(float) * n) != cudaSuccess ||
        cudaMemset(sp->gate, 0, sizeof(float) * n) != cudaSuccess)
      return sfail(sp, SPH_E_CUDA, "clearing the species failed");
  }
  return SPH_OK;
}

void sph_species_destroy(sph_species* sp) {
  if (!sp) return;
  cudaFree(sp->by_row);
  cudaFree(sp->r0);
  cudaFree(sp->r1);
  cudaFree(sp->vol);
  cudaFree(sp->nonuniform);
  cudaFree(sp->gate);
  cudaFree(sp->scale_by_row);
  cudaFree(sp->sq);
  cudaFree(sp->stage);
  cudaFree(sp->Bc);
  cudaFree(sp->Lrow);
  cudaFree(sp->Lc);
  delete sp;
}

const char* sph_species_last_error(const sph_species* sp) { return sp ? sp->err.c_str() : "null species"; }

}  // extern "C"

namespace {

int species_upload(sph_handle* h, sph_species* sp, const double* C, float* dst, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (sp->n == 0) return SPH_OK;
  if (!C) return sfail(sp, SPH_E_INVALID, "the array is required");
  cudaStream_t s = (cudaStream_t)stream;
  const double* src = C;
  const PtrKind kind = pointer_kind(C);
  if (kind == kOtherDevicePtr) return sfail(sp, SPH_E_INVALID, "the array lives on another device");
  if (kind == kHostPtr) {
    if (cudaMemcpyAsync(sp->stage, C, sizeof(double) * sp->n, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return sfail(sp, SPH_E_CUDA, "copy of the species failed");
    src = sp->stage;
  }
  sph::k_species_import<<<sph::diff_grid(sp->n), sph::kDiffBlock, 0, s>>>(sp->n, src, dst);
  ++h->launches;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "species upload failed");
  return SPH_OK;
}

int species_download(sph_handle* h, sph_species* sp, const float* src, double* C, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (sp->n == 0) return SPH_OK;
  if (!C) return sfail(sp, SPH_E_INVALID, "the array is required");
  cudaStream_t s = (cudaStream_t)stream;
  const PtrKind kind = pointer_kind(C);
  if (kind == kOtherDevicePtr) return sfail(sp, SPH_E_INVALID, "the array lives on another device");
  const bool dev = kind == kDevicePtr;
  double* dst = dev ? C : sp->stage;
  sph::k_species_export<<<sph::diff_grid(sp->n), sph::kDiffBlock, 0, s>>>(sp->n, src, dst);
  ++h->launches;
  if (!dev && cudaMemcpyAsync(C, sp->stage, sizeof(double) * sp->n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "copy of the species failed");
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "species download failed");
  return SPH_OK;
}

}  // namespace

extern "C" {

int sph_species_set(sph_handle* h, sph_species* sp, const double* C, void* stream) {
  return species_upload(h, sp, C, sp ? sp->by_row : nullptr, stream);
}

int sph_species_get(sph_handle* h, sph_species* sp, double* C, void* stream) {
  return species_download(h, sp, sp ? sp->by_row : nullptr, C, stream);
}

int sph_species_set_gate(sph_handle* h, sph_species* sp, const double* w, void* stream) {
  return species_upload(h, sp, w, sp ? sp->gate : nullptr, stream);
}

int sph_species_get_gate(sph_handle* h, sph_species* sp, double* w, void* stream) {
  return species_download(h, sp, sp ? sp->gate : nullptr, w, stream);
}

int sph_species_set_scale(sph_handle* h, sph_species* sp, const double* s, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (sp->n == 0) return SPH_OK;
  if (!sp->scale_by_row) {
    if (cudaMalloc(&sp->scale_by_row, sizeof(float) * sp->n) != cudaSuccess ||
        cudaMalloc(&sp->sq, sizeof(float) * sp->n) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(sp->scale_by_row);
      sp->scale_by_row = nullptr;
      return sfail(sp, SPH_E_OOM, "device allocation of the diffusivity factors failed");
    }
  }
  // any failure from here on leaves the species with no factors, as before the first call
  auto drop_factors = [sp](int code, const char* msg) {
    cudaFree(sp->scale_by_row);
    cudaFree(sp->sq);
    sp->scale_by_row = nullptr;
    sp->sq = nullptr;
    if (msg) sp->err = msg;
    return code;
  };
  int r = species_upload(h, sp, s, sp->scale_by_row, stream);
  if (r != SPH_OK) return drop_factors(r, nullptr);
  cudaStream_t st = (cudaStream_t)stream;
  int bad = 0;
  if (cudaMemsetAsync(sp->nonuniform, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return drop_factors(SPH_E_CUDA, "check failed");
  }
  sph::k_check_scale<<<sph::diff_grid(sp->n), sph::kDiffBlock, 0, st>>>(sp->n, sp->scale_by_row, sp->nonuniform);
  ++h->launches;
  if (cudaMemcpyAsync(&bad, sp->nonuniform, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return drop_factors(SPH_E_CUDA, "check failed");
  }
  if (bad) return drop_factors(SPH_E_INVALID, "diffusivity factors must be positive and finite");
  return SPH_OK;
}

int sph_species_set_tensors(sph_handle* h, sph_species* sp, const double* Dp, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (!Dp) {                       // back to the species' own tensor
    cudaFree(sp->Lrow);
    cudaFree(sp->Lc);
    sp->Lrow = nullptr;
    sp->Lc = nullptr;
    return SPH_OK;
  }
  if (sp->n == 0) return SPH_OK;
  const PtrKind kind = pointer_kind(Dp);
  if (kind == kOtherDevicePtr) return sfail(sp, SPH_E_INVALID, "the array lives on another device");
  cudaStream_t st = (cudaStream_t)stream;
  const int d = sp->dim;
  const size_t n = (size_t)sp->n, nd = n * d * d;
  float* Lrow = nullptr;
  float4* Lc = nullptr;
  double* staged = nullptr;
  auto cleanup = [&](int code, const char* msg) {
    cudaGetLastError();
    cudaFree(Lrow);
    cudaFree(Lc);
    cudaFree(staged);
    return sfail(sp, code, msg);
  };
  if (cudaMalloc(&Lrow, sizeof(float) * 6 * n) != cudaSuccess ||
      cudaMalloc(&Lc, sizeof(float4) * n * (d == 2 ? 1 : 2)) != cudaSuccess)
    return cleanup(SPH_E_OOM, "device allocation of the tensor factors failed");
  const double* src = Dp;
  if (kind == kHostPtr) {
    if (cudaMalloc(&staged, sizeof(double) * nd) != cudaSuccess)
      return cleanup(SPH_E_OOM, "staging allocation of the tensors failed");
    if (cudaMemcpyAsync(staged, Dp, sizeof(double) * nd, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return cleanup(SPH_E_CUDA, "copy of the tensors failed");
    src = staged;
  }
  int bad = 0;
  if (cudaMemsetAsync(sp->nonuniform, 0, sizeof(int), st) != cudaSuccess)
    return cleanup(SPH_E_CUDA, "tensor set-up failed");
  sph::k_species_factor<<<sph::diff_grid(sp->n), sph::kDiffBlock, 0, st>>>(sp->n, d, src, Lrow, sp->nonuniform);
  ++h->launches;
  if (cudaMemcpyAsync(&bad, sp->nonuniform, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cleanup(SPH_E_CUDA, "tensor set-up failed");
  if (bad) return cleanup(SPH_E_INVALID, "every D_i must be finite, symmetric and positive definite");
  cudaFree(staged);
  cudaFree(sp->Lrow);
  cudaFree(sp->Lc);
  sp->Lrow = Lrow;
  sp->Lc = Lc;
  return SPH_OK;
}

int sph_species_set_correction(sph_handle* h, sph_species* sp, int32_t on) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (on && !sp->Bc && sp->n > 0) {
    if (cudaMalloc(&sp->Bc, sizeof(float4) * (size_t)sp->n * (sp->dim == 2 ? 1 : 2)) != cudaSuccess) {
      cudaGetLastError();
      sp->Bc = nullptr;
      return sfail(sp, SPH_E_OOM, "device allocation of the correction matrices failed");
    }
  }
  sp->corrected = on != 0;
  return SPH_OK;
}

int sph_reaction_step(sph_handle* h, sph_species* sp, const sph_reaction* r, double dt, int32_t n_steps,
                      void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (!r || (r->model != SPH_REACTION_FN && r->model != SPH_REACTION_AP))
    return sfail(sp, SPH_E_INVALID, "unknown reaction model");
  const double vals[] = {r->a, r->b, r->k, r->eps0, r->mu1, r->mu2, r->beta, r->gamma, r->sigma};
  for (double v : vals)
    if (!std::isfinite(v)) return sfail(sp, SPH_E_INVALID, "reaction parameters must be finite");
  if (!(std::isfinite(dt) && dt > 0.0) || n_steps < 0) return sfail(sp, SPH_E_INVALID, "dt must be > 0 and n_steps >= 0");
  if (sp->n == 0 || n_steps == 0) return SPH_OK;
  const sph::ReactCoef R{r->model, (float)r->a, (float)r->b, (float)r->k, (float)r->eps0, (float)r->mu1,
                         (float)r->mu2, (float)r->beta, (float)r->gamma, (float)r->sigma};
  cudaStream_t s = (cudaStream_t)stream;
  sph::k_reaction<<<sph::diff_grid(sp->n), sph::kDiffBlock, 0, s>>>(sp->n, sp->by_row, sp->gate, R, (float)dt,
                                                                    n_steps);
  ++h->launches;
  if (cudaGetLastError() != cudaSuccess) return sfail(sp, SPH_E_CUDA, "reaction launch failed");
  return SPH_OK;
}

int sph_diffusion_step(sph_handle* h, sph_species* sp, double dt, int32_t n_steps, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (!(std::isfinite(dt) && dt > 0.0) || n_steps < 0) return sfail(sp, SPH_E_INVALID, "dt must be > 0 and n_steps >= 0");
  if (!h->cells_valid) return sfail(sp, SPH_E_INVALID, "sph_build_cells must run after a state change");
  {
    const int r = sph_debug_check(h, (cudaStream_t)stream);
    if (r != SPH_OK) return sfail(sp, r, "neighbour table check failed (SPH_FLAG_DEBUG_BOUNDS)");
  }
  const sph::Buffers& b = h->b;
  if (b.n == 0 || n_steps == 0) return SPH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = sph::diff_grid(b.n);
  const float fdt = (float)dt;
  if (cudaMemsetAsync(sp->nonuniform, 0, sizeof(int), s) != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "diffusion set-up failed");
  auto pack = b.dim == 2 ? sph::k_species_pack<2> : sph::k_species_pack<3>;
  pack<<<grid, sph::kDiffBlock, 0, s>>>(b.n, b.PS, b.id, b.inst_of, b.inst, b.mass, sp->by_row, sp->r0,
                                        sp->r1, sp->vol, sp->scale_by_row, sp->sq, sp->nonuniform);
  // the one synchronisation of the call: which stage kernels the volumes and factors allow
  int nonuniform = 0;
  if (cudaMemcpyAsync(&nonuniform, sp->nonuniform, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "diffusion set-up failed");
  const bool ten = sp->Lrow != nullptr;
  const bool unif = nonuniform == 0 && !ten;
  sph::StageFn s1, s2;
  if (b.dim == 2) {
    if (b.any_periodic) sph::pick_stages<2, true>(sp->iso, unif, sp->corrected, ten, &s1, &s2);
    else sph::pick_stages<2, false>(sp->iso, unif, sp->corrected, ten, &s1, &s2);
  } else {
    if (b.any_periodic) sph::pick_stages<3, true>(sp->iso, unif, sp->corrected, ten, &s1, &s2);
    else sph::pick_stages<3, false>(sp->iso, unif, sp->corrected, ten, &s1, &s2);
  }
  if (ten) {                       // the tensor factors per slot (sqrt(s) folded in)
    auto pt = b.dim == 2 ? sph::k_species_pack_tensors<2> : sph::k_species_pack_tensors<3>;
    pt<<<grid, sph::kDiffBlock, 0, s>>>(b.n, b.id, sp->Lrow, sp->scale_by_row, sp->Lc);
    ++h->launches;
  }
  const float* sq_stage = ten ? nullptr : sp->sq;
  if (sp->corrected) {             // B0 of the current configuration, once per call
    auto corr = b.dim == 2 ? (b.any_periodic ? sph::k_species_correction<2, true> : sph::k_species_correction<2, false>)
                           : (b.any_periodic ? sph::k_species_correction<3, true> : sph::k_species_correction<3, false>);
    corr<<<grid, sph::kDiffBlock, 0, s>>>(b.n, sp->r0, b.nbr, b.nbc, b.inst_of, b.inst, sp->vol, sp->Bc);
    ++h->launches;
  }
  for (int k = 0; k < n_steps; ++k) {
    s1<<<grid, sph::kDiffBlock, 0, s>>>(b.n, sp->r0, sp->r1, b.nbr, b.nbc, b.inst_of, b.inst, sp->vol,
                                         sq_stage, sp->K, fdt, sp->Bc, sp->Lc);
    s2<<<grid, sph::kDiffBlock, 0, s>>>(b.n, sp->r1, sp->r0, b.nbr, b.nbc, b.inst_of, b.inst, sp->vol,
                                         sq_stage, sp->K, fdt, sp->Bc, sp->Lc);
  }
  sph::k_species_unpack<<<grid, sph::kDiffBlock, 0, s>>>(b.n, b.id, sp->r0, sp->by_row);
  h->launches += 2 + 2 * (int64_t)n_steps;
  if (cudaGetLastError() != cudaSuccess) return sfail(sp, SPH_E_CUDA, "diffusion launch failed");
  return SPH_OK;
}

}  // extern "C"
