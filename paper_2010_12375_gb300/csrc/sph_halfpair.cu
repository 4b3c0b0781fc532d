// Symmetric half-pair evaluation of the two relaxations (Newton's third law): every
// unordered fluid pair of the frozen neighbour set is evaluated once.
//
// The pair terms split into a part both particles share and a sign:
//   momentum (Eq. riemannsph):  dv_i/dt -= m_j Q_ij,  dv_j/dt += m_i Q_ij,
//                               Q_ij = 2 P*_ij (dW/dr)/r r_ij / (rho_i rho_j)
//     (P*_ij = P*_ji, and the kernel gradient is antisymmetric: the weak form of
//      Eq. gradsph-weak, whose antisymmetry is what conserves momentum);
//   continuity:                 drho_i/dt += 2 rho_i V_j (h_ij + c_ij) dW/dr,
//                               drho_j/dt += 2 rho_j V_i (h_ij - c_ij) dW/dr,
//     h_ij = (v_i - v_j).r_ij / (2|r_ij|) (the velocity part of U* - U_L, symmetric),
//     c_ij = c0 (rho_i - rho_j) / (rho_i + rho_j) (its pressure part, antisymmetric).
// Pass A: particle i takes every neighbour j > i (in storage order), adds its own share to
// registers and stores j's share in a per-slot buffer at (slot of j in i's row, i). Pass B:
// particle j adds the shares stored for it by every neighbour i < j, found through a
// reverse-slot map built once per configuration update (slot of j in i's row, for every
// slot of j's row holding an i < j), then its wall pairs, and finishes the update exactly as
// the per-pair kernels do. Sums run in a fixed order and there are no atomics, so the
// result is bit-reproducible; it differs from the per-pair kernels only by rounding.
//
// Walls are one-sided (static) and stay with the fluid particle, in pass B. Not combined
// with the frozen geometry or the transport velocity; one thread per particle.
#include "sph_relax.cuh"

namespace sph {
namespace {

constexpr int kHBlock = 128;

inline unsigned hgrid(int64_t n) { return (unsigned)((n + kHBlock - 1) / kHBlock); }

// Reverse slots: for slot t of particle j holding i < j, the slot of j in i's fluid row.
// Rows are in ascending storage order when no axis is periodic (the search visits cells in
// flattened order), so a binary search finds it; periodic rows are searched linearly.
template <bool PER>
__global__ void __launch_bounds__(kHBlock)
k_reverse_slots(int64_t n, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc, uint8_t* __restrict__ rev,
                Global* g) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int nf = (int)(nbc[j] & 0xffffu);
  for (int t = 0; t < nf; ++t) {
    const int i = nbr[slot_index(n, j, t)];
    if ((int64_t)i >= j) continue;
    const int ni = (int)(nbc[i] & 0xffffu);
    int found = -1;
    if (!PER) {
      int lo = 0, hi = ni - 1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = nbr[slot_index(n, i, mid)];
        if ((int64_t)v == j) { found = mid; break; }
        if ((int64_t)v < j) lo = mid + 1;
        else hi = mid - 1;
      }
    } else {
      for (int s = 0; s < ni; ++s)
        if ((int64_t)nbr[slot_index(n, i, s)] == j) { found = s; break; }
    }
    if (found < 0) {              // the relation is symmetric by construction; never expected
      atomicOr(&g->err, ERR_BOUNDS);
      found = 0;
    }
    rev[(int64_t)t * n + j] = (uint8_t)found;
  }
}

template <bool PER>
__device__ __forceinline__ float axis_diff(int qi, int qj, int period, float dq, float add) {
  return fmaf(biased_diff<PER>(qi, qj, period) - kMagic, dq, add);
}

// ---------------------------------------------------------------- pressure relaxation --
template <int D, bool PER, bool UNI>
__global__ void __launch_bounds__(kHBlock)
k_pr_half_a(const Inst Ip, int64_t n, const int4* __restrict__ PS, const float4* __restrict__ VS,
            const float* __restrict__ mass, const int* __restrict__ inst_of, const Inst* __restrict__ inst,
            const Ctrl* __restrict__ ctrl, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
            float4* __restrict__ share, float4* __restrict__ part) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = inst_index(inst_of, i);
  const double dtd = ctrl[k].dt;
  if (dtd == 0.0) return;
  const Inst& I = UNI ? Ip : inst[k];
  const float hdt = 0.5f * (float)dtd;
  const int4 pi = PS[i];
  const float4 vi = VS[i];
  const float dev_i = i2f(pi.w) + hdt * vi.w;
  const float rho_i = I.rho0 + dev_i;
  const float m_i = mass ? mass[i] : I.mass;
  const int px = PER ? I.period[0] : 0, py = PER ? I.period[1] : 0, pz = PER ? I.period[2] : 0;
  const int nf = (int)(nbc[i] & 0xffffu);
  float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
  for (int s = 0; s < nf; ++s) {
    const int j = nbr[slot_index(n, i, s)];
    if ((int64_t)j <= i) continue;
    const int4 pj = PS[j];
    const float4 vj = VS[j];
    const float dvx = vj.x - vi.x, dvy = vj.y - vi.y, dvz = D == 3 ? vj.z - vi.z : 0.f;
    const float rx = axis_diff<PER>(pi.x, pj.x, px, I.dq, -hdt * dvx);
    const float ry = axis_diff<PER>(pi.y, pj.y, py, I.dq, -hdt * dvy);
    const float rz = D == 3 ? axis_diff<PER>(pi.z, pj.z, pz, I.dq, -hdt * dvz) : 0.f;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, kTinyR2)));
    const float inv_r = rsqrtf(r2);
    const float t = fmaxf(fmaf(r2 * inv_r, -0.5f * I.inv_h, 1.0f), 0.0f);
    const float fw = I.dwr_a * t * t * t;
    const float dev_j = fmaf(hdt, vj.w, i2f(pj.w));
    const float rho_j = I.rho0 + dev_j;
    const float dU = (dvx * rx + dvy * ry + dvz * rz) * inv_r;
    const float beta = fminf(I.kc * fmaxf(dU, 0.0f), 1.0f);
    const float pstar = fmaf(I.qc0 * (rho_i + rho_j), beta * dU, I.hc0sq * (dev_i + dev_j));
    const float q = 2.0f * pstar * fw * __fdividef(1.0f, rho_i * rho_j);
    const float m_j = mass ? mass[j] : I.mass;
    kahan_add(sx, cx, -m_j * q * rx);
    kahan_add(sy, cy, -m_j * q * ry);
    if (D == 3) kahan_add(sz, cz, -m_j * q * rz);
    share[(int64_t)s * n + i] = make_float4(m_i * q * rx, m_i * q * ry, m_i * q * rz, 0.f);
  }
  part[i] = make_float4(sx - cx, sy - cy, sz - cz, 0.f);
}

template <int D, bool PER, bool UNI>
__global__ void __launch_bounds__(kHBlock)
k_pr_half_b(const Inst Ip, int64_t n, const int4* __restrict__ PS, const float4* __restrict__ VS,
            int4* __restrict__ PH, float4* __restrict__ VH, const int* __restrict__ inst_of,
            const Inst* __restrict__ inst, Ctrl* ctrl, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
            const uint8_t* __restrict__ rev, const float4* __restrict__ share, const float4* __restrict__ part,
            const int4* __restrict__ WP, const float4* __restrict__ WN, const float4* __restrict__ acc_prior,
            float4* __restrict__ acc_keep, Global* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int kb;
  const bool uni = block_one_instance<1>(inst_of, n, &kb);
  bool valid = i < n;
  const int k = valid ? inst_index(inst_of, i) : kb;
  const double dtd = ctrl[k].dt;
  if (dtd == 0.0) valid = false;
  const Inst& I = UNI ? Ip : inst[k];
  float v2 = 0.f;
  if (valid) {
    const float dt = (float)dtd;
    PrCtx C;
    C.sx = C.sy = C.sz = C.nx = C.ny = C.nz = f2(0.f);
    C.hdt = 0.5f * dt;
    C.px = PER ? I.period[0] : 0;
    C.py = PER ? I.period[1] : 0;
    C.pz = PER ? I.period[2] : 0;
    const int4 pi = PS[i];
    const float4 vi = VS[i];
    C.dev_i = i2f(pi.w) + C.hdt * vi.w;
    C.rho_i = I.rho0 + C.dev_i;
    C.pr_i = I.c0sq * C.dev_i;
    const uint32_t cnt = nbc[i];
    const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
    // shares stored for this particle by its neighbours below it
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (int t = 0; t < nf; ++t) {
      const int j = nbr[slot_index(n, i, t)];
      if ((int64_t)j >= i) continue;
      const int s = rev[(int64_t)t * n + i];
      const float4 q = share[(int64_t)s * n + j];
      kahan_add(sx, cx, q.x);
      kahan_add(sy, cy, q.y);
      if (D == 3) kahan_add(sz, cz, q.z);
    }
    if (nw) {                     // walls: the per-pair kernel's packed wall terms
      const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
      const float2 DQ = f2(I.dq);
      const int q0 = wall_slot0(nf) >> 2, nwq = (nw + 3) >> 2;
      for (int q = 0; q < nwq; ++q) {
        const int4 c = nb4[(int64_t)(q0 + q) * n + i];
        const int s = q << 2;
        const int w1 = s + 1 < nw ? c.y : c.x, w2 = s + 2 < nw ? c.z : c.x, w3 = s + 3 < nw ? c.w : c.x;
        const int4 a0 = WP[c.x], a1 = WP[w1], a2 = WP[w2], a3 = WP[w3];
        const float4 n0 = WN[c.x], n1 = WN[w1], n2 = WN[w2], n3 = WN[w3];
        const float2 V01 = make_float2(i2f(a0.w), s + 1 < nw ? i2f(a1.w) : 0.0f);
        const float2 V23 = make_float2(s + 2 < nw ? i2f(a2.w) : 0.0f, s + 3 < nw ? i2f(a3.w) : 0.0f);
        pr_wall2<D, PER>(I, C, pi, vi, a0, a1, n0, n1, V01, DQ);
        pr_wall2<D, PER>(I, C, pi, vi, a2, a3, n2, n3, V23, DQ);
      }
    }
    const float sc = -2.0f / C.rho_i;
    const float wx = (C.sx.x + C.nx.x) + (C.sx.y + C.nx.y);
    const float wy = (C.sy.x + C.ny.x) + (C.sy.y + C.ny.y);
    const float wz = (C.sz.x + C.nz.x) + (C.sz.y + C.nz.y);
    const float4 up = part[i];
    const float4 ap = acc_prior ? acc_prior[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float a0 = ap.x + I.g[0] + sc * wx + (up.x + (sx - cx));
    const float a1 = ap.y + I.g[1] + sc * wy + (up.y + (sy - cy));
    const float a2 = D == 3 ? ap.z + I.g[2] + sc * wz + (up.z + (sz - cz)) : 0.f;
    const float4 vn = make_float4(vi.x + dt * a0, vi.y + dt * a1, vi.z + dt * a2, vi.w);
    const float hdt = C.hdt;
    int qx = pi.x + __float2int_rn(hdt * vi.x * I.inv_dq);
    int qy = pi.y + __float2int_rn(hdt * vi.y * I.inv_dq);
    int qz = D == 3 ? pi.z + __float2int_rn(hdt * vi.z * I.inv_dq) : 0;
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
  reduce_vmax(v2, valid, k, uni, ctrl);
}

// ---------------------------------------------------------------- density relaxation ---
template <int D, bool PER, bool UNI>
__global__ void __launch_bounds__(kHBlock)
k_dr_half_a(const Inst Ip, int64_t n, const int4* __restrict__ PH, const float4* __restrict__ VH,
            const float* __restrict__ mass, const int* __restrict__ inst_of, const Inst* __restrict__ inst,
            const Ctrl* __restrict__ ctrl, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
            float* __restrict__ share, float* __restrict__ part) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = inst_index(inst_of, i);
  const double dtd = ctrl[k].dt;
  if (dtd == 0.0) return;
  const Inst& I = UNI ? Ip : inst[k];
  const float hdt = 0.5f * (float)dtd;
  const int4 pi = PH[i];
  const float4 vi = VH[i];
  const float dev_i = i2f(pi.w);
  const float rho_i = I.rho0 + dev_i;
  const float V_i = (mass ? mass[i] : I.mass) / rho_i;
  const int px = PER ? I.period[0] : 0, py = PER ? I.period[1] : 0, pz = PER ? I.period[2] : 0;
  const int nf = (int)(nbc[i] & 0xffffu);
  float sum = 0.f, comp = 0.f;
  for (int s = 0; s < nf; ++s) {
    const int j = nbr[slot_index(n, i, s)];
    if ((int64_t)j <= i) continue;
    const int4 pj = PH[j];
    const float4 vj = VH[j];
    const float dvx = vi.x - vj.x, dvy = vi.y - vj.y, dvz = D == 3 ? vi.z - vj.z : 0.f;
    const float rx = axis_diff<PER>(pi.x, pj.x, px, I.dq, hdt * dvx);
    const float ry = axis_diff<PER>(pi.y, pj.y, py, I.dq, hdt * dvy);
    const float rz = D == 3 ? axis_diff<PER>(pi.z, pj.z, pz, I.dq, hdt * dvz) : 0.f;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, kTinyR2)));
    const float inv_r = rsqrtf(r2);
    const float r = r2 * inv_r;
    const float t = fmaxf(fmaf(r, -0.5f * I.inv_h, 1.0f), 0.0f);
    const float dW = I.dwr_a * t * t * t * r;                 // dW/dr
    const float dev_j = i2f(pj.w);
    const float rho_j = I.rho0 + dev_j;
    const float h = (dvx * rx + dvy * ry + dvz * rz) * inv_r * 0.5f;
    const float c = I.c0 * (dev_i - dev_j) * __fdividef(1.0f, rho_i + rho_j);
    const float V_j = (mass ? mass[j] : I.mass) / rho_j;
    kahan_add(sum, comp, V_j * (h + c) * dW);
    share[(int64_t)s * n + i] = V_i * (h - c) * dW;
  }
  part[i] = sum - comp;
}

template <int D, bool PER, bool UNI>
__global__ void __launch_bounds__(kHBlock)
k_dr_half_b(const Inst Ip, int64_t n, const int4* __restrict__ PH, const float4* __restrict__ VH,
            int4* __restrict__ PS, float4* __restrict__ VS, const int* __restrict__ inst_of,
            const Inst* __restrict__ inst, const Ctrl* __restrict__ ctrl, const int* __restrict__ nbr,
            const uint32_t* __restrict__ nbc, const uint8_t* __restrict__ rev, const float* __restrict__ share,
            const float* __restrict__ part, const int4* __restrict__ WP, const float4* __restrict__ WN, Global* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = inst_index(inst_of, i);
  const double dtd = ctrl[k].dt;
  if (dtd == 0.0) return;
  const Inst& I = UNI ? Ip : inst[k];
  DrCtx C;
  C.s = C.nc = f2(0.f);
  C.hdt = 0.5f * (float)dtd;
  C.px = PER ? I.period[0] : 0;
  C.py = PER ? I.period[1] : 0;
  C.pz = PER ? I.period[2] : 0;
  const int4 pi = PH[i];
  const float4 vi = VH[i];
  C.dev_i = i2f(pi.w);
  C.rho_i = I.rho0 + C.dev_i;
  const uint32_t cnt = nbc[i];
  const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
  float sum = 0.f, comp = 0.f;
  for (int t = 0; t < nf; ++t) {
    const int j = nbr[slot_index(n, i, t)];
    if ((int64_t)j >= i) continue;
    kahan_add(sum, comp, share[(int64_t)rev[(int64_t)t * n + i] * n + j]);
  }
  if (nw) {
    const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
    const float2 DQ = f2(I.dq);
    const float pr_i = I.c0sq * C.dev_i;
    const int q0 = wall_slot0(nf) >> 2, nwq = (nw + 3) >> 2;
    for (int q = 0; q < nwq; ++q) {
      const int4 c = nb4[(int64_t)(q0 + q) * n + i];
      const int s = q << 2;
      const int w1 = s + 1 < nw ? c.y : c.x, w2 = s + 2 < nw ? c.z : c.x, w3 = s + 3 < nw ? c.w : c.x;
      const int4 a0 = WP[c.x], a1 = WP[w1], a2 = WP[w2], a3 = WP[w3];
      const float4 n0 = WN[c.x], n1 = WN[w1], n2 = WN[w2], n3 = WN[w3];
      const float2 V01 = make_float2(i2f(a0.w), s + 1 < nw ? i2f(a1.w) : 0.0f);
      const float2 V23 = make_float2(s + 2 < nw ? i2f(a2.w) : 0.0f, s + 3 < nw ? i2f(a3.w) : 0.0f);
      dr_wall2<D, PER>(I, C, pi, vi, a0, a1, n0, n1, V01, DQ, pr_i);
      dr_wall2<D, PER>(I, C, pi, vi, a2, a3, n2, n3, V23, DQ, pr_i);
    }
  }
  const float walls = (C.s.x + C.nc.x) + (C.s.y + C.nc.y);
  const float drho = 2.0f * C.rho_i * (walls + (part[i] + (sum - comp)));
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

template <int D, bool PER, bool UNI>
void launch_half_t(const Buffers& b, bool pressure, cudaStream_t s) {
  const unsigned grid = hgrid(b.n);
  const int4* wp = b.nw ? b.WP : nullptr;
  const float4* wn = b.nw ? b.WN : nullptr;
  if (pressure) {
    k_pr_half_a<D, PER, UNI><<<grid, kHBlock, 0, s>>>(b.inst0, b.n, b.PS, b.VS, b.mass, b.inst_of, b.inst, b.ctrl,
                                                      b.nbr, b.nbc, b.hshare, b.hpart);
    k_pr_half_b<D, PER, UNI><<<grid, kHBlock, 0, s>>>(b.inst0, b.n, b.PS, b.VS, b.PH, b.VH, b.inst_of, b.inst, b.ctrl,
                                                      b.nbr, b.nbc, b.hrev, b.hshare, b.hpart, wp, wn, b.acc_prior,
                                                      b.acc_keep, b.glob);
  } else {
    float* share = reinterpret_cast<float*>(b.hshare);
    float* part = reinterpret_cast<float*>(b.hpart);
    k_dr_half_a<D, PER, UNI><<<grid, kHBlock, 0, s>>>(b.inst0, b.n, b.PH, b.VH, b.mass, b.inst_of, b.inst, b.ctrl,
                                                      b.nbr, b.nbc, share, part);
    k_dr_half_b<D, PER, UNI><<<grid, kHBlock, 0, s>>>(b.inst0, b.n, b.PH, b.VH, b.PS, b.VS, b.inst_of, b.inst, b.ctrl,
                                                      b.nbr, b.nbc, b.hrev, share, part, wp, wn, b.glob);
  }
}

template <int D, bool PER>
void launch_half_d(const Buffers& b, bool pressure, cudaStream_t s) {
  if (b.n_inst == 1) launch_half_t<D, PER, true>(b, pressure, s);
  else launch_half_t<D, PER, false>(b, pressure, s);
}

}  // namespace

void launch_reverse_slots(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0 || !b.hrev) return;
  if (b.any_periodic) k_reverse_slots<true><<<hgrid(b.n), kHBlock, 0, s>>>(b.n, b.nbr, b.nbc, b.hrev, b.glob);
  else k_reverse_slots<false><<<hgrid(b.n), kHBlock, 0, s>>>(b.n, b.nbr, b.nbc, b.hrev, b.glob);
  ++*launches;
}

void launch_half_pair(const Buffers& b, bool pressure, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  if (b.dim == 2) {
    if (b.any_periodic) launch_half_d<2, true>(b, pressure, s);
    else launch_half_d<2, false>(b, pressure, s);
  } else {
    if (b.any_periodic) launch_half_d<3, true>(b, pressure, s);
    else launch_half_d<3, false>(b, pressure, s);
  }
  *launches += 2;
}

}  // namespace sph
