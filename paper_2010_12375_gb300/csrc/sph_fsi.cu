// Multi-resolution fluid-structure coupling (paper Sec. "Multi-resolution FSI coupling",
// "Total Lagrangian formulation", "Position-based Verlet scheme"): an elastic solid of its
// own resolution (spacing, smoothing length h_S) coupled to the fluid of a single-tank handle.
//
// Solid (total Lagrangian): neighbours fixed in the reference configuration, with the
// reference kernel gradient grad0_a W_ab = dW/dr r0_ab/|r0_ab| (the true gradient) and the
// correction matrix B0_a = (sum_b V_b (r0_b - r0_a) (x) grad0_a W_ab)^-1 (Eq. sph-correctmatrix),
// both computed once, in FP64. A solid step (Eqs. verlet-first-half-solid,
// verlet-first-mediate-solid, verlet-first-final-solid): F += dt/2 dF/dt, r += dt/2 v, first
// Piola-Kirchhoff stress P = F S (linear elastic: S = lambda tr E I + 2 mu E; Neo-Hookean:
// S = mu (I - C^-1) + lambda ln J C^-1), dv/dt = (2/m_a) sum_b V_a V_b P~_ab grad0_a W_ab + g +
// f_a/m_a with P~_ab = (P_a B0_a + P_b B0_b)/2 (Eq. sph-mechanical-mom), v += dt dv/dt,
// r += dt/2 v, dF/dt = (sum_b V_b (v_b - v_a) (x) grad0_a W_ab) B0_a, F += dt/2 dF/dt.
// Clamped particles keep their reference position and zero velocity.
//
// Coupling, per fluid acoustic step of length dt_F (the fluid kernel h_F throughout):
//  * after the fluid pressure relaxation, every fluid particle near the solid adds
//    f_i/m_i to its new velocity, f_i = sum_a -2 V_i V_a pbar grad_i W(r_ia) (Eq. fs-force-mr-sp),
//    pbar = (p_i rho^d + p^d rho_i)/(rho_i + rho^d), with the imaginary pressure
//    p^d = p_i + rho_i max(0, -(g - a~_a).n_a) ((r_i - r_a).n_a) (Eq. fs-coupling-mr read as the
//    hydrostatic extrapolation, n_a the solid's normal into the fluid), plus, with viscosity,
//    2 eta V_i V_a (v_i - v^d)/(|r| + 0.01 h) dW/dr, v^d = 2 v~_a - v_i (Eq. fs-force-mr-sv);
//    the solid takes the opposite force, summed per solid particle with the same pair
//    function, so the two are equal and opposite bit for bit; the fluid's |v|max is then
//    recomputed;
//  * after the fluid density relaxation, each near fluid particle adds the continuity term
//    of its solid neighbours as moving walls (U_L = -n.v_i, U_R = -U_L - 2 n.v~_a, P_R = p^d);
//  * then kappa = [dt_F/dt_S] + 1 solid steps of dt_F/kappa (dt_S of Eq. dts-advection) with
//    the fluid force held, in one thread-block cluster; v~ and a~ become their averages.
// The fluid particles near the solid (inside its bounding box widened by 3 h_F) are listed
// once per configuration update, in storage order.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "sph.h"
#include "sph_handle.h"
#include "sph_kernels.h"

namespace sph {
namespace {

namespace cg = cooperative_groups;

constexpr int kFBlock = 128;
constexpr int kSolidThreads = 1024;       // threads per block of the solid-step cluster
constexpr int kMaxSolid = 16 * kSolidThreads;
constexpr int kMaxSolidSteps = 1 << 16;   // solid steps in one fluid step, at most

inline unsigned fgrid(int64_t n) { return (unsigned)((n + kFBlock - 1) / kFBlock); }
// blocks for a warp per item over up to n items: 16 blocks an SM at most (grid-stride beyond)
inline unsigned wgrid(int64_t n) {
  constexpr int w = kFBlock / 32;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + w - 1) / w, 152 * 16));
}

struct SolidMat {
  int model, dim;
  int single_step;                        // cap the fluid's next acoustic step at dt_S
  float lam, mu, rho0;
  double h, c;                            // smoothing length and sound speed sqrt(K / rho0)
  float g[3];
};

// d x d matrices stored element-major: M[(r * d + c) * ns + a]; D is a compile-time
// dimension so the small matrices stay in registers
template <int D>
__device__ __forceinline__ void load_mat(const float* M, int64_t ns, int64_t a, float m[D * D]) {
#pragma unroll
  for (int k = 0; k < D * D; ++k) m[k] = M[(int64_t)k * ns + a];
}
template <int D>
__device__ __forceinline__ void store_mat(float* M, int64_t ns, int64_t a, const float m[D * D]) {
#pragma unroll
  for (int k = 0; k < D * D; ++k) M[(int64_t)k * ns + a] = m[k];
}

// ---------------------------------------------------------------- reference set-up ------
// Neighbour slots as (owning block << 16) | slot in its tile, once the cluster's particles
// per block P is fixed: the solid steps then address a neighbour's shared memory directly.
__global__ void k_solid_pack_rows(int64_t ns, int cap, const int* __restrict__ cnt, int P, int* __restrict__ nb) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  const int c = min(cnt[a], cap);
  for (int t = 0; t < c; ++t) {
    const int b = nb[(int64_t)t * ns + a];
    nb[(int64_t)t * ns + a] = ((b / P) << 16) | (b % P);
  }
}

// One thread per solid particle: its neighbours within 2 h_S in the reference configuration
// (ascending index), their kernel gradients times the neighbour's volume gV_ab = V_b grad0_a
// W_ab, the row sum c_a = sum_b gV_ab, and B0 (all in FP64, then stored in FP32).
__global__ void k_solid_setup(int64_t ns, int d, double h, const double* __restrict__ x0,
                              const double* __restrict__ vol, int cap, int* __restrict__ nb,
                              int* __restrict__ cnt, float4* __restrict__ gV, float4* __restrict__ cA,
                              float* __restrict__ B0, int* err) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  const double pi = 3.14159265358979323846;
  const double alpha = d == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
  double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double csum[3] = {0, 0, 0};
  int c = 0;
  for (int64_t b = 0; b < ns; ++b) {
    if (b == a) continue;
    double r[3] = {0, 0, 0}, r2 = 0;
    for (int k = 0; k < d; ++k) {
      r[k] = x0[a * d + k] - x0[b * d + k];
      r2 += r[k] * r[k];
    }
    if (!(r2 < 4.0 * h * h)) continue;
    if (c >= cap) {
      atomicOr(err, 1);
      continue;
    }
    const double dist = sqrt(r2), q = dist / h, t = 1.0 - 0.5 * q;
    const double fw = alpha / h * (-5.0 * q) * t * t * t / dist;     // (dW/dr) / r
    double g[3] = {fw * r[0], fw * r[1], fw * r[2]};
    nb[(int64_t)c * ns + a] = (int)b;
    gV[(int64_t)c * ns + a] = make_float4((float)(vol[b] * g[0]), (float)(vol[b] * g[1]), (float)(vol[b] * g[2]), 0.f);
    for (int k = 0; k < 3; ++k) csum[k] += vol[b] * g[k];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) M[i * d + j] += vol[b] * (-r[i]) * g[j];   // (r0_b - r0_a) (x) grad
    ++c;
  }
  cnt[a] = c;
  cA[a] = make_float4((float)csum[0], (float)csum[1], (float)csum[2], 0.f);
  double inv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (d == 2) {
    const double det = M[0] * M[3] - M[1] * M[2];
    inv[0] = M[3] / det; inv[1] = -M[1] / det; inv[2] = -M[2] / det; inv[3] = M[0] / det;
  } else {
    const double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                       M[2] * (M[3] * M[7] - M[4] * M[6]);
    inv[0] = (M[4] * M[8] - M[5] * M[7]) / det; inv[1] = (M[2] * M[7] - M[1] * M[8]) / det;
    inv[2] = (M[1] * M[5] - M[2] * M[4]) / det; inv[3] = (M[5] * M[6] - M[3] * M[8]) / det;
    inv[4] = (M[0] * M[8] - M[2] * M[6]) / det; inv[5] = (M[2] * M[3] - M[0] * M[5]) / det;
    inv[6] = (M[3] * M[7] - M[4] * M[6]) / det; inv[7] = (M[1] * M[6] - M[0] * M[7]) / det;
    inv[8] = (M[0] * M[4] - M[1] * M[3]) / det;
  }
  for (int k = 0; k < d * d; ++k) {
    if (!isfinite(inv[k])) atomicOr(err, 2);
    B0[(int64_t)k * ns + a] = (float)inv[k];
  }
}

// ---------------------------------------------------------------- near-fluid list -------
__global__ void k_solid_bbox(int64_t ns, const int4* __restrict__ X, int pad, int* __restrict__ box) {
  __shared__ int lo[3][kSolidThreads / 32], hi[3][kSolidThreads / 32];
  int l[3] = {INT_MAX, INT_MAX, INT_MAX}, u[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int64_t a = threadIdx.x; a < ns; a += blockDim.x) {
    const int4 q = X[a];
    const int v[3] = {q.x, q.y, q.z};
    for (int k = 0; k < 3; ++k) {
      l[k] = min(l[k], v[k]);
      u[k] = max(u[k], v[k]);
    }
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      l[k] = min(l[k], __shfl_xor_sync(0xffffffffu, l[k], o));
      u[k] = max(u[k], __shfl_xor_sync(0xffffffffu, u[k], o));
    }
    if ((threadIdx.x & 31) == 0) {
      lo[k][threadIdx.x >> 5] = l[k];
      hi[k][threadIdx.x >> 5] = u[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int k = threadIdx.x;
    int a = INT_MAX, b = INT_MIN;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a = min(a, lo[k][w]);
      b = max(b, hi[k][w]);
    }
    box[k] = a > INT_MIN + pad ? a - pad : INT_MIN;
    box[3 + k] = b < INT_MAX - pad ? b + pad : INT_MAX;
  }
}

__global__ void k_near_flags(int64_t n, int d, const int4* __restrict__ PS, const int* __restrict__ box,
                             uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 p = PS[i];
  bool in = p.x >= box[0] && p.x <= box[3] && p.y >= box[1] && p.y <= box[4];
  if (d == 3) in = in && p.z >= box[2] && p.z <= box[5];
  flag[i] = in ? 1u : 0u;
}

// The list in storage order, and its length (kept on the device, so a captured graph reads
// each configuration update's own length).
__global__ void k_near_compact(int64_t n, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ off,
                               int* __restrict__ near, int* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) near[off[i]] = (int)i;
  if (i == n - 1) *count = (int)(off[i] + flag[i]);
}

// ---------------------------------------------------------------- coupling pair terms ---
struct FsiPair {
  float rx, ry, rz, r, dW;
  bool in;
};

template <int D>
__device__ __forceinline__ FsiPair fsi_geometry(const int4& qi, const int4& qa, const Inst& I) {
  FsiPair P;
  const int dx = qi.x - qa.x, dy = qi.y - qa.y, dz = D == 3 ? qi.z - qa.z : 0;
  const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
  P.in = d2 < I.R2;
  P.rx = (float)dx * I.dq;
  P.ry = (float)dy * I.dq;
  P.rz = (float)dz * I.dq;
  P.r = sqrtf(P.rx * P.rx + P.ry * P.ry + P.rz * P.rz);
  P.dW = kernel_dW_over_r(P.r, I) * P.r;                  // dW/dr
  return P;
}

// p^d of Eq. fs-coupling-mr (hydrostatic extrapolation with the solid's mean acceleration)
__device__ __forceinline__ float imaginary_pressure(float p_i, float rho_i, const FsiPair& P, const float4& n,
                                                    const float4& abar, const Inst& I) {
  const float proj = fmaxf(0.0f, -((I.g[0] - abar.x) * n.x + (I.g[1] - abar.y) * n.y + (I.g[2] - abar.z) * n.z));
  return p_i + rho_i * proj * (P.rx * n.x + P.ry * n.y + P.rz * n.z);
}

// Force on fluid particle i from solid particle a (pressure and, with viscosity, viscous):
// the same function on both sides, so action and reaction agree bit for bit.
__device__ __forceinline__ float3 fsi_force(const FsiPair& P, float dev_i, float m_i, const float4& v_i,
                                            float V_a, const float4& n, const float4& vbar, const float4& abar,
                                            const Inst& I) {
  const float rho_i = I.rho0 + dev_i;
  const float p_i = I.c0sq * dev_i;
  const float pd = imaginary_pressure(p_i, rho_i, P, n, abar, I);
  const float rhod = I.rho0 + pd * I.inv_c0sq;
  const float pbar = (p_i * rhod + pd * rho_i) / (rho_i + rhod);
  const float V_i = m_i / rho_i;
  const float fw = P.r > 0.0f ? P.dW / P.r : 0.0f;
  const float cp = -2.0f * V_i * V_a * pbar * fw;
  float3 f = make_float3(cp * P.rx, cp * P.ry, cp * P.rz);
  if (I.eta > 0.0f) {
    // v_i - v^d = 2 (v_i - v~_a)
    const float cv = 2.0f * I.eta * V_i * V_a / (P.r + 0.01f * I.h) * P.dW * 2.0f;
    f.x += cv * (v_i.x - vbar.x);
    f.y += cv * (v_i.y - vbar.y);
    f.z += cv * (v_i.z - vbar.z);
  }
  return f;
}

// The coupling sums run a warp per particle. The other side's particles come in chunks of
// 32 consecutive ones (the solid in its Morton order, the near fluid list in storage order)
// with the bounding box of their current positions: the warp tests 32 boxes at a time and
// visits only chunks whose box lies within 2h (the box distance bounds every pair distance
// from below, so no pair is missed), each lane taking one particle of a visited chunk with
// a compensated running sum; the warp combines the 32 shares by a fixed shuffle tree of
// error-free sums, so every result is deterministic. The grids are fixed (a grid-stride loop
// over warps), since the near list's length is on the device.
constexpr int kCoupleWarps = kFBlock / 32;

// Bounding box (lo, hi) of the positions of each chunk of 32 consecutive entries of a list
// (idx[k], or k itself when idx is NULL) of n entries, n on the device when n_dev is given.
__global__ void __launch_bounds__(kFBlock)
k_chunk_boxes(int64_t n_host, const int* __restrict__ n_dev, const int* __restrict__ idx, const int4* __restrict__ X,
              int4* __restrict__ box) {
  const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
  const int lane = threadIdx.x & 31;
  for (int64_t c = (int64_t)blockIdx.x * kCoupleWarps + (threadIdx.x >> 5); c * 32 < n;
       c += (int64_t)gridDim.x * kCoupleWarps) {
    const int64_t k = c * 32 + lane;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (k < n) {
      const int4 q = X[idx ? (int64_t)idx[k] : k];
      lo[0] = hi[0] = q.x;
      lo[1] = hi[1] = q.y;
      lo[2] = hi[2] = q.z;
    }
    for (int a = 0; a < 3; ++a) {
      lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
      hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
    }
    if (lane == 0) {
      box[2 * c] = make_int4(lo[0], lo[1], lo[2], 0);
      box[2 * c + 1] = make_int4(hi[0], hi[1], hi[2], 0);
    }
  }
}

// Whether a chunk's box comes within the support of q: the squared distance from q to the
// box (in position quanta) below the pair threshold R2.
template <int D>
__device__ __forceinline__ bool box_within(const int4& q, const int4& lo, const int4& hi, long long R2) {
  const long long dx = max(max((long long)lo.x - q.x, (long long)q.x - hi.x), 0LL);
  const long long dy = max(max((long long)lo.y - q.y, (long long)q.y - hi.y), 0LL);
  const long long dz = D == 3 ? max(max((long long)lo.z - q.z, (long long)q.z - hi.z), 0LL) : 0LL;
  return dx * dx + dy * dy + dz * dz < R2;
}

// Error-free sum of two floats (Knuth's two-sum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Running sum with its error term, and the warp-wide combination of 32 such pairs.
__device__ __forceinline__ void csum_add(float& s, float& e, float x) {
  float t;
  two_sum(s, x, s, t);
  e += t;
}
__device__ __forceinline__ float csum_warp(float s, float e) {
  for (int o = 16; o > 0; o >>= 1) {
    const float so = __shfl_xor_sync(0xffffffffu, s, o), eo = __shfl_xor_sync(0xffffffffu, e, o);
    float t;
    two_sum(s, so, s, t);
    e += eo + t;
  }
  return s + e;
}

template <int D>
__global__ void __launch_bounds__(kFBlock)
k_fsi_fluid_pressure(const Inst I, const int* __restrict__ n_near_p, const int* __restrict__ near, const int4* __restrict__ PH,
                     float4* __restrict__ VH, const float4* __restrict__ VS, const float* __restrict__ mass,
                     const Ctrl* __restrict__ ctrl, int64_t ns, const int4* __restrict__ X,
                     const float4* __restrict__ N, const float4* __restrict__ vbar, const float4* __restrict__ abar,
                     const int4* __restrict__ sbox, float4* __restrict__ acc_keep) {
  const double dtd = ctrl[0].dt;
  if (dtd == 0.0) return;
  const int lane = threadIdx.x & 31;
  const int n_near = *n_near_p;
  const int64_t nch = (ns + 31) / 32;
  for (int k = blockIdx.x * kCoupleWarps + (threadIdx.x >> 5); k < n_near; k += gridDim.x * kCoupleWarps) {
    const int i = near[k];
    const int4 qi = PH[i];
    const float dev_i = i2f(qi.w);
    const float m_i = mass ? mass[i] : I.mass;
    const float4 vi = VS[i];
    float s[3] = {0, 0, 0}, e[3] = {0, 0, 0};
    for (int64_t c0 = 0; c0 < nch; c0 += 32) {
      const int64_t c = c0 + lane;
      unsigned hits = __ballot_sync(0xffffffffu, c < nch && box_within<D>(qi, sbox[2 * c], sbox[2 * c + 1], I.R2));
      while (hits) {
        const int64_t a = (c0 + __ffs(hits) - 1) * 32 + lane;
        hits &= hits - 1;
        if (a >= ns) continue;
        const int4 qa = X[a];
        const FsiPair P = fsi_geometry<D>(qi, qa, I);
        if (!P.in) continue;
        const float3 f = fsi_force(P, dev_i, m_i, vi, i2f(qa.w), N[a], vbar[a], abar[a], I);
        csum_add(s[0], e[0], f.x / m_i);
        csum_add(s[1], e[1], f.y / m_i);
        if (D == 3) csum_add(s[2], e[2], f.z / m_i);
      }
    }
    const float ax = csum_warp(s[0], e[0]), ay = csum_warp(s[1], e[1]), az = D == 3 ? csum_warp(s[2], e[2]) : 0.f;
    if (lane == 0) {
      const float dt = (float)dtd;
      float4 v = VH[i];
      v.x += dt * ax;
      v.y += dt * ay;
      if (D == 3) v.z += dt * az;
      VH[i] = v;
      if (acc_keep) {
        float4 acc = acc_keep[i];
        acc.x += ax;
        acc.y += ay;
        acc.z += az;
        acc_keep[i] = acc;
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kFBlock)
k_fsi_solid_force(const Inst I, const int* __restrict__ n_near_p, const int* __restrict__ near, const int4* __restrict__ PH,
                  const float4* __restrict__ VS, const float* __restrict__ mass, const Ctrl* __restrict__ ctrl,
                  int64_t ns, const int4* __restrict__ X, const float4* __restrict__ N,
                  const float4* __restrict__ vbar, const float4* __restrict__ abar, const int4* __restrict__ fbox,
                  float4* __restrict__ force) {
  if (ctrl[0].dt == 0.0) return;
  const int lane = threadIdx.x & 31;
  const int n_near = *n_near_p;
  const int nch = (n_near + 31) / 32;
  for (int64_t a = (int64_t)blockIdx.x * kCoupleWarps + (threadIdx.x >> 5); a < ns; a += (int64_t)gridDim.x * kCoupleWarps) {
    const int4 qa = X[a];
    const float V_a = i2f(qa.w);
    const float4 n = N[a], vb = vbar[a], ab = abar[a];
    float s[3] = {0, 0, 0}, e[3] = {0, 0, 0};
    for (int c0 = 0; c0 < nch; c0 += 32) {
      const int c = c0 + lane;
      unsigned hits = __ballot_sync(0xffffffffu, c < nch && box_within<D>(qa, fbox[2 * c], fbox[2 * c + 1], I.R2));
      while (hits) {
        const int k = (c0 + __ffs(hits) - 1) * 32 + lane;
        hits &= hits - 1;
        if (k >= n_near) continue;
        const int i = near[k];
        const int4 qi = PH[i];
        const FsiPair P = fsi_geometry<D>(qi, qa, I);
        if (!P.in) continue;
        const float m_i = mass ? mass[i] : I.mass;
        const float3 f = fsi_force(P, i2f(qi.w), m_i, VS[i], V_a, n, vb, ab, I);
        csum_add(s[0], e[0], -f.x);
        csum_add(s[1], e[1], -f.y);
        if (D == 3) csum_add(s[2], e[2], -f.z);
      }
    }
    const float fx = csum_warp(s[0], e[0]), fy = csum_warp(s[1], e[1]), fz = D == 3 ? csum_warp(s[2], e[2]) : 0.f;
    if (lane == 0) force[a] = make_float4(fx, fy, fz, 0.f);
  }
}

template <int D>
__global__ void __launch_bounds__(kFBlock)
k_fsi_fluid_continuity(const Inst I, const int* __restrict__ n_near_p, const int* __restrict__ near, int4* __restrict__ PS,
                       float4* __restrict__ VS, const int4* __restrict__ PH, const Ctrl* __restrict__ ctrl,
                       int64_t ns, const int4* __restrict__ X, const float4* __restrict__ N,
                       const float4* __restrict__ vbar, const float4* __restrict__ abar, const int4* __restrict__ sbox) {
  const double dtd = ctrl[0].dt;
  if (dtd == 0.0) return;
  const int lane = threadIdx.x & 31;
  const int n_near = *n_near_p;
  const int64_t nch = (ns + 31) / 32;
  for (int k = blockIdx.x * kCoupleWarps + (threadIdx.x >> 5); k < n_near; k += gridDim.x * kCoupleWarps) {
    const int i = near[k];
    int4 qi = PS[i];                       // r^{n+1}, and the new density deviation in w
    float4 vi = VS[i];                     // v^{n+1}
    const float dev_h = i2f(PH[i].w);      // rho_i is the mid-point density, as in the fluid pass
    const float rho_i = I.rho0 + dev_h;
    const float p_i = I.c0sq * dev_h;
    float s = 0.f, e = 0.f;
    for (int64_t c0 = 0; c0 < nch; c0 += 32) {
      const int64_t c = c0 + lane;
      unsigned hits = __ballot_sync(0xffffffffu, c < nch && box_within<D>(qi, sbox[2 * c], sbox[2 * c + 1], I.R2));
      while (hits) {
        const int64_t a = (c0 + __ffs(hits) - 1) * 32 + lane;
        hits &= hits - 1;
        if (a >= ns) continue;
        const int4 qa = X[a];
        const FsiPair P = fsi_geometry<D>(qi, qa, I);
        if (!P.in) continue;
        const float4 n = N[a], vb = vbar[a];
        const float UL = -(n.x * vi.x + n.y * vi.y + n.z * vi.z);
        const float uw = -(n.x * vb.x + n.y * vb.y + n.z * vb.z);
        const float UR = -UL + 2.0f * uw;
        const float PR = imaginary_pressure(p_i, rho_i, P, n, abar[a], I);
        const float rhoR = I.rho0 + PR * I.inv_c0sq;
        const float Us = 0.5f * (UL + UR) + (p_i - PR) / ((rho_i + rhoR) * I.c0);   // (P_L - P_R)/(2 rho_bar c0)
        csum_add(s, e, 2.0f * rho_i * i2f(qa.w) * (Us - UL) * P.dW);
      }
    }
    const float drho = csum_warp(s, e);
    if (lane == 0) {
      const float hdt = 0.5f * (float)dtd;
      qi.w = f2i(i2f(qi.w) + hdt * drho);
      vi.w += drho;
      PS[i] = qi;
      VS[i] = vi;
    }
  }
}

// ---------------------------------------------------------------- solid steps ----------
// First Piola-Kirchhoff stress from the displacement gradient H = F - I (what the solid
// stores: near the reference configuration F - I carries the strain without the
// cancellation that forming F^T F - I in FP32 would cost). K = C - I = H + H^T + H^T H.
//   linear:       E = K/2, S = lambda tr(E) I + 2 mu E
//   Neo-Hookean:  S = mu (I - C^-1) + lambda ln J C^-1 = C^-1 (mu K + lambda ln J I),
//                 ln J = log1p(det(I + H) - 1) with the determinant expanded in H
// P = F S = S + H S.
template <int D>
__device__ __forceinline__ void first_piola(const SolidMat& M, const float H[D * D], float P[D * D]) {
  constexpr int d = D;
  float K[9];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      float s = H[i * d + j] + H[j * d + i];
      for (int k = 0; k < d; ++k) s += H[k * d + i] * H[k * d + j];
      K[i * d + j] = s;
    }
  float S[9];
  if (M.model == SPH_SOLID_LINEAR) {
    float trE = 0.f;
    for (int i = 0; i < d; ++i) trE += 0.5f * K[i * d + i];
    for (int i = 0; i < d * d; ++i) S[i] = M.mu * K[i];
    for (int i = 0; i < d; ++i) S[i * d + i] += M.lam * trE;
  } else {
    float C[9], Ci[9], detC, Jm1;
    for (int i = 0; i < d * d; ++i) C[i] = K[i];
    for (int i = 0; i < d; ++i) C[i * d + i] += 1.0f;
    if (d == 2) {
      detC = C[0] * C[3] - C[1] * C[2];
      Ci[0] = C[3] / detC; Ci[1] = -C[1] / detC; Ci[2] = -C[2] / detC; Ci[3] = C[0] / detC;
      Jm1 = H[0] + H[3] + (H[0] * H[3] - H[1] * H[2]);
    } else {
      detC = C[0] * (C[4] * C[8] - C[5] * C[7]) - C[1] * (C[3] * C[8] - C[5] * C[6]) + C[2] * (C[3] * C[7] - C[4] * C[6]);
      Ci[0] = (C[4] * C[8] - C[5] * C[7]) / detC; Ci[1] = (C[2] * C[7] - C[1] * C[8]) / detC;
      Ci[2] = (C[1] * C[5] - C[2] * C[4]) / detC; Ci[3] = (C[5] * C[6] - C[3] * C[8]) / detC;
      Ci[4] = (C[0] * C[8] - C[2] * C[6]) / detC; Ci[5] = (C[2] * C[3] - C[0] * C[5]) / detC;
      Ci[6] = (C[3] * C[7] - C[4] * C[6]) / detC; Ci[7] = (C[1] * C[6] - C[0] * C[7]) / detC;
      Ci[8] = (C[0] * C[4] - C[1] * C[3]) / detC;
      const float tr = H[0] + H[4] + H[8];
      const float minors = (H[0] * H[4] - H[1] * H[3]) + (H[0] * H[8] - H[2] * H[6]) + (H[4] * H[8] - H[5] * H[7]);
      const float detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                         H[2] * (H[3] * H[7] - H[4] * H[6]);
      Jm1 = tr + minors + detH;
    }
    const float lnJ = log1pf(Jm1);
    float A[9];
    for (int i = 0; i < d * d; ++i) A[i] = M.mu * K[i];
    for (int i = 0; i < d; ++i) A[i * d + i] += M.lam * lnJ;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        float s = 0.f;
        for (int k = 0; k < d; ++k) s += Ci[i * d + k] * A[k * d + j];
        S[i * d + j] = s;
      }
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      float s = S[i * d + j];
      for (int k = 0; k < d; ++k) s += H[i * d + k] * S[k * d + j];
      P[i * d + j] = s;
    }
}

struct SolidPtrs {
  int64_t ns;
  int4* X;
  float4* V;
  const uint8_t* fixed;
  const float* vol;      // reference volumes
  float *F, *dFdt;       // F: the displacement gradient H = F - I
  const float* B0;
  const int* nb;         // neighbour slots, packed (block << 16) | tile slot
  const int* cnt;
  const float4* gV;      // V_b grad0_a W_ab per slot
  const float4* cA;      // sum_b V_b grad0_a W_ab per particle
  const float4* force;
  float4 *acc, *vbar, *abar;
  long long* steps;      // solid steps taken, total
  int* kappa_last;
  double* dt_cap;        // the fluid's cap (single time stepping), or NULL
  Global* g;             // the handle's error word
  int lanes;             // lanes per particle in the neighbour sums: 1, 2, 4, 8, 16 or 32
  int per_block;         // particles owned by each block of the cluster (the last may own fewer)
  int row;               // slots a particle in the staged rows (the longest reference row)
};

// Shared-memory image of the particles one block owns during the solid steps: what the
// neighbours read (P B0 as D rows of a float4 each -- one float4 in 2D --, and v) and the
// owner's own state. Bytes per particle: 80 + 16 R + 8 D^2, R = 1 (2D) or 3 (3D).
__host__ __device__ constexpr int pb_rows(int d) { return d == 2 ? 1 : 3; }
template <int D>
struct SolidTile {
  float4* V;             // published: velocity
  float4* PB;            // published: P B0, rows [l * R + r]
  int4* X;               // position (fixed point) and volume bits
  float4 *acc, *vsum, *asum;
  float *F, *dF;         // H = F - I and dF/dt, element-major [k * P + l]
  __device__ SolidTile(void* base, int P) {
    float4* f4 = reinterpret_cast<float4*>(base);
    V = f4;
    PB = f4 + P;
    X = reinterpret_cast<int4*>(PB + pb_rows(D) * P);
    acc = reinterpret_cast<float4*>(X + P);
    vsum = acc + P;
    asum = vsum + P;
    F = reinterpret_cast<float*>(asum + P);
    dF = F + D * D * P;
  }
};
__host__ __device__ constexpr int solid_tile_bytes(int d, int P) {
  return (P * (80 + 16 * pb_rows(d) + 8 * d * d) + 15) / 16 * 16;   // what follows stays 16-byte aligned
}

// P B0 of tile slot l as a d x d matrix (2D: one float4 holds the four entries)
template <int D>
__device__ __forceinline__ void load_pb(const float4* PB, int l, float m[D * D]) {
  if (D == 2) {
    const float4 r = PB[l];
    m[0] = r.x; m[1] = r.y; m[2] = r.z; m[3] = r.w;
  } else {
    for (int i = 0; i < D; ++i) {
      const float4 r = PB[l * 3 + i];
      m[i * D] = r.x;
      m[i * D + 1] = r.y;
      m[i * D + 2] = r.z;
    }
  }
}
template <int D>
__device__ __forceinline__ void store_pb(float4* PB, int l, const float m[D * D]) {
  if (D == 2) PB[l] = make_float4(m[0], m[1], m[2], m[3]);
  else
    for (int i = 0; i < D; ++i) PB[l * 3 + i] = make_float4(m[i * D], m[i * D + 1], m[i * D + 2], 0.f);
}

// Largest |v|^2 and |dv/dt|^2 over the solid, the same in every thread of the cluster:
// per block through shared memory, then each block reads the others' through distributed
// shared memory. Ends with a cluster barrier, so the per-block slots can be reused.
__device__ __forceinline__ void cluster_vmax(cg::cluster_group& cl, float& vm, float& am, float (*red)[kSolidThreads / 32],
                                             float* blk) {
  for (int o = 16; o > 0; o >>= 1) {
    vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = vm;
    red[1][threadIdx.x >> 5] = am;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      vm = fmaxf(vm, red[0][w]);
      am = fmaxf(am, red[1][w]);
    }
    blk[0] = vm;
    blk[1] = am;
  }
  cl.sync();
  if (threadIdx.x == 0) {
    for (unsigned r = 0; r < cl.num_blocks(); ++r) {
      const float* o = cl.map_shared_rank(blk, r);
      vm = fmaxf(vm, o[0]);
      am = fmaxf(am, o[1]);
    }
    red[0][0] = vm;
    red[1][0] = am;
  }
  cl.sync();                               // every block has read every other block's slots
  vm = red[0][0];
  am = red[1][0];
}

__device__ __forceinline__ bool gt_is_first() { return threadIdx.x == 0 && blockIdx.x == 0; }

// Eq. dts-advection from the largest |v|^2 and |dv/dt|^2 (CFL 0.6).
__device__ __forceinline__ double solid_dt(const SolidMat& M, float vm, float am) {
  double dts = M.h / (M.c + sqrt((double)vm));
  if (am > 0.f) dts = fmin(dts, sqrt(M.h / sqrt((double)am)));
  return 0.6 * dts;
}

// The constant data of the solid steps: per-slot neighbour rows (packed owner slots, V_b
// grad0 W) and per-particle counts, c_a, fluid force, volume, B0 and clamp flags. Read from
// global memory (particle a, slot t at [t ns + a]), or with CS staged once per launch into
// the block's shared memory after the tile (tile slot l, slot t at [l row + t]): the cluster
// barrier's acquire drops L1, so global reads would go to L2 on every phase.
template <int D, bool CS>
struct SolidConst {
  const int* nb;
  const float4* gV;
  const int* cnt;
  const float4 *cA, *force;
  const float* vol;
  const float* B0;
  const uint8_t* fixed;
  int64_t ss, ps, bs;    // slot stride, particle stride of the rows, element stride of B0
  __device__ int slot(int64_t p, int t) const { return CS ? nb[t * ss + p * ps] : __ldg(nb + t * ss + p * ps); }
  __device__ float4 grad(int64_t p, int t) const { return CS ? gV[t * ss + p * ps] : __ldg(gV + t * ss + p * ps); }
  __device__ int count(int64_t p) const { return CS ? cnt[p] : __ldg(cnt + p); }
  __device__ float4 csum(int64_t p) const { return CS ? cA[p] : __ldg(cA + p); }
  __device__ float4 f(int64_t p) const { return CS ? force[p] : __ldg(force + p); }
  __device__ float v(int64_t p) const { return CS ? vol[p] : __ldg(vol + p); }
  __device__ float b0(int64_t p, int k) const { return CS ? B0[k * bs + p] : __ldg(B0 + k * bs + p); }
  __device__ bool clamped(int64_t p) const { return (CS ? fixed[p] : __ldg(fixed + p)) != 0; }
};

// Shared-memory bytes per particle of the staged constants (row slots a particle): the rows
// (16 + 4 bytes a slot), c_a and the fluid force (16 each), count and volume (4 each), B0
// (4 d^2) and the clamp flag (1)
__host__ __device__ constexpr int solid_const_bytes(int d, int row) { return row * 20 + 40 + 4 * d * d + 1; }

// First half of a solid step for the owned particle at tile slot l, whose F (the H = F - I
// of the end of the last step) and dF/dt the caller holds: F += dt/2 dF/dt, r += dt/2 v,
// and P B0 published for the neighbours' stress divergence.
template <int D, bool CS>
__device__ __forceinline__ void solid_first_half(const Inst& I, const SolidMat& M, const SolidConst<D, CS>& C,
                                                 int64_t p, const SolidTile<D>& T, int P, int l, float F[D * D],
                                                 const float dF[D * D], float hh) {
  constexpr int d = D;
  for (int k = 0; k < d * d; ++k) {
    F[k] += hh * dF[k];
    T.F[k * P + l] = F[k];
  }
  if (!C.clamped(p)) {
    const float4 v = T.V[l];
    int4 q = T.X[l];
    q.x += __float2int_rn(hh * v.x * I.inv_dq);
    q.y += __float2int_rn(hh * v.y * I.inv_dq);
    if (d == 3) q.z += __float2int_rn(hh * v.z * I.inv_dq);
    T.X[l] = q;
  }
  float Pk[D * D], B[D * D], PB[D * D];
  first_piola<D>(M, F, Pk);
#pragma unroll
  for (int k = 0; k < d * d; ++k) B[k] = C.b0(p, k);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      float s = 0.f;
      for (int k = 0; k < d; ++k) s += Pk[i * d + k] * B[k * d + j];
      PB[i * d + j] = s;
    }
  store_pb<D>(T.PB, l, PB);
}

// All kappa solid steps of one fluid acoustic step in one thread-block cluster (up to 16
// blocks of up to 1024 threads: as many as the owned particles' lane groups need), the
// solid held in the cluster's distributed shared memory: block
// r owns the particles [r P, (r + 1) P) (internal order: a Morton curve of the reference
// positions) and keeps their state, and with CS the constant rows too, in its shared
// memory for the whole launch; global memory is read at the start and written at the end.
// A neighbour's P B0 and v are read from its owner's shared memory. Each owned particle
// belongs to a group of `lanes` adjacent lanes: its first lane updates the particle's
// state, the others take strided shares of its reference neighbours, combined by a shuffle
// tree (plain FP32 sums: compensated ones moved no parity figure and cost 2 % of the step).
// Two phases a step, each ended by a cluster barrier:
//   A. dv/dt from the neighbours' P B0, then v and the second half of r;
//   B. dF/dt = (sum_b V_b (v_b - v_a) (x) grad0 W) B0 from the neighbours' new v, F to the
//      end of the step, and straight on the next step's first half (F, r, P B0).
// kappa is computed identically in every block. A step that is not positive and finite, or
// more than kMaxSolidSteps solid steps in one fluid step, sets ERR_DT and takes no step.
template <int D, bool CS>
__global__ void __launch_bounds__(kSolidThreads, 1)
k_solid_steps(const Inst I, SolidMat M, SolidPtrs S, const Ctrl* __restrict__ ctrl) {
  cg::cluster_group cl = cg::this_cluster();
  const double dtF = ctrl[0].dt;           // the same in every block
  if (dtF == 0.0) return;
  if (S.lanes < 1 || S.lanes > 32 || (S.lanes & (S.lanes - 1)) != 0 || S.per_block < 1 ||
      (int64_t)S.per_block * cl.num_blocks() < S.ns || (CS && S.row < 1)) {   // the host sizes these
    if (gt_is_first() && S.g) atomicOr(&S.g->err, ERR_BOUNDS);
    return;
  }
  constexpr int d = D;
  extern __shared__ float4 tile_mem[];
  const int P = S.per_block;
  const unsigned rank = cl.block_rank();
  const SolidTile<D> T(tile_mem, P);
  const int64_t first = (int64_t)rank * P;
  const int own = (int)max((int64_t)0, min((int64_t)P, S.ns - first));   // particles this block owns
  const int L = S.lanes;                   // divides 32: a group never spans two warps
  const int lane = (int)(threadIdx.x & (unsigned)(L - 1));
  const int gpb = (int)blockDim.x / L, grp = (int)threadIdx.x / L;
  __shared__ float red[2][kSolidThreads / 32];
  __shared__ float blk[2];
  __shared__ int s_kappa;

  // the constants: global, or staged after the tile
  SolidConst<D, CS> C;
  if (CS) {
    const int row = S.row;
    char* base = reinterpret_cast<char*>(tile_mem) + solid_tile_bytes(d, P);
    float4* gVs = reinterpret_cast<float4*>(base);
    float4* cAs = gVs + (int64_t)P * row;
    float4* fs = cAs + P;
    int* nbs = reinterpret_cast<int*>(fs + P);
    int* cnts = nbs + (int64_t)P * row;
    float* vols = reinterpret_cast<float*>(cnts + P);
    float* B0s = vols + P;
    uint8_t* fxs = reinterpret_cast<uint8_t*>(B0s + d * d * P);
    for (int l = threadIdx.x; l < own; l += blockDim.x) {
      const int64_t a = first + l;
      cnts[l] = min(S.cnt[a], row);
      cAs[l] = S.cA[a];
      fs[l] = S.force[a];
      vols[l] = S.vol[a];
      fxs[l] = S.fixed[a];
      for (int k = 0; k < d * d; ++k) B0s[k * P + l] = S.B0[(int64_t)k * S.ns + a];
    }
    for (int64_t idx = threadIdx.x; idx < (int64_t)own * row; idx += blockDim.x) {
      const int t = (int)(idx / own), l = (int)(idx - (int64_t)t * own);
      const int64_t a = first + l;
      if (t < S.cnt[a]) {
        nbs[(int64_t)l * row + t] = S.nb[(int64_t)t * S.ns + a];
        gVs[(int64_t)l * row + t] = S.gV[(int64_t)t * S.ns + a];
      }
    }
    C = SolidConst<D, CS>{nbs, gVs, cnts, cAs, fs, vols, B0s, fxs, 1, row, P};
  } else {
    C = SolidConst<D, CS>{S.nb, S.gV, S.cnt, S.cA, S.force, S.vol, S.B0, S.fixed, S.ns, 1, S.ns};
  }
  // index of particle (tile slot l) in the constants
  auto cp = [&](int l) -> int64_t { return CS ? (int64_t)l : first + l; };

  // the owned particles into shared memory; Eq. dts-advection from the state at the start
  // of the fluid step (R25)
  float vm = 0.f, am = 0.f;
  for (int l = threadIdx.x; l < own; l += blockDim.x) {
    const int64_t a = first + l;
    const float4 v = S.V[a], ac = S.acc[a];
    T.V[l] = v;
    T.X[l] = S.X[a];
    T.acc[l] = ac;
    T.vsum[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    T.asum[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < d * d; ++k) {
      T.F[k * P + l] = S.F[(int64_t)k * S.ns + a];
      T.dF[k * P + l] = S.dFdt[(int64_t)k * S.ns + a];
    }
    vm = fmaxf(vm, v.x * v.x + v.y * v.y + v.z * v.z);
    am = fmaxf(am, ac.x * ac.x + ac.y * ac.y + ac.z * ac.z);
  }
  cluster_vmax(cl, vm, am, red, blk);      // also orders the staging above for the whole block
  if (threadIdx.x == 0) {
    const double dts = solid_dt(M, vm, am);
    const double r = dtF / dts;
    int kappa = 0;
    if (dts > 0.0 && r < (double)kMaxSolidSteps) kappa = (int)floor(r) + 1;
    else if (rank == 0 && S.g) atomicOr(&S.g->err, ERR_DT);
    s_kappa = kappa;
    if (rank == 0) {
      *S.kappa_last = kappa;
      *S.steps += kappa;
    }
  }
  __syncthreads();
  const int kappa = s_kappa;
  if (kappa == 0) return;                  // the same decision in every block; nothing written
  const double hd = dtF / kappa;
  const float h = (float)hd, hh = 0.5f * h;
  for (int l = threadIdx.x; l < own; l += blockDim.x) {
    float F[D * D], dF[D * D];
    for (int k = 0; k < d * d; ++k) {
      F[k] = T.F[k * P + l];
      dF[k] = T.dF[k * P + l];
    }
    solid_first_half<D, CS>(I, M, C, cp(l), T, P, l, F, dF, hh);
  }
  cl.sync();
  for (int step = 0; step < kappa; ++step) {
    // A: dv/dt, v, r the second half (passes uniform over the block for the shuffles). With
    // gV_ab = V_b grad0 W and c_a = sum_b gV_ab, Eq. sph-mechanical-mom's sum
    // (2 / m_a) sum_b V_a V_b (P_a B0_a + P_b B0_b)/2 grad0 W = (P_a B0_a c_a + sum_b P_b B0_b gV_ab) / rho0.
    for (int base = 0; base < own; base += gpb) {
      const int l = base + grp;
      const bool live = l < own;
      const int64_t p = cp(l);
      const bool moves = live && !C.clamped(p);
      float sx[3] = {0.f, 0.f, 0.f};
      if (moves) {
        const int nc = C.count(p);
#pragma unroll 2
        for (int t = lane; t < nc; t += L) {
          const int pk = C.slot(p, t);
          const float4 g = C.grad(p, t);
          const float gv[3] = {g.x, g.y, g.z};
          float PBb[D * D];
          load_pb<D>(cl.map_shared_rank(T.PB, (unsigned)(pk >> 16)), pk & 0xffff, PBb);
          for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) sx[i] = fmaf(PBb[i * d + j], gv[j], sx[i]);
        }
      }
      for (int o = L >> 1; o > 0; o >>= 1)
        for (int i = 0; i < d; ++i) sx[i] += __shfl_xor_sync(0xffffffffu, sx[i], o);
      if (live && lane == 0) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 v = T.V[l];
        if (moves) {
          float PBa[D * D];
          load_pb<D>(T.PB, l, PBa);
          const float4 c4 = C.csum(p);
          const float cv[3] = {c4.x, c4.y, c4.z};
          float div[3] = {0.f, 0.f, 0.f};
          for (int i = 0; i < d; ++i) {
            float y = 0.0f;
            for (int j = 0; j < d; ++j) y = fmaf(PBa[i * d + j], cv[j], y);
            div[i] = sx[i] + y;
          }
          const float inv_rho0 = 1.0f / M.rho0, inv_m = inv_rho0 / C.v(p);
          const float4 f = C.f(p);
          acc.x = div[0] * inv_rho0 + M.g[0] + f.x * inv_m;
          acc.y = div[1] * inv_rho0 + M.g[1] + f.y * inv_m;
          acc.z = d == 3 ? div[2] * inv_rho0 + M.g[2] + f.z * inv_m : 0.f;
          v.x += h * acc.x;
          v.y += h * acc.y;
          v.z += h * acc.z;
          T.V[l] = v;
          int4 q = T.X[l];
          q.x += __float2int_rn(hh * v.x * I.inv_dq);
          q.y += __float2int_rn(hh * v.y * I.inv_dq);
          if (d == 3) q.z += __float2int_rn(hh * v.z * I.inv_dq);
          T.X[l] = q;
        }
        T.acc[l] = acc;
        float4 vs = T.vsum[l], as = T.asum[l];
        vs.x += v.x; vs.y += v.y; vs.z += v.z;
        as.x += acc.x; as.y += acc.y; as.z += acc.z;
        T.vsum[l] = vs;
        T.asum[l] = as;
      }
    }
    cl.sync();                             // v published; every read of P B0 done
    // B: dF/dt from the new velocities, F the second half, then the next step's first half
    const bool more = step + 1 < kappa;
    for (int base = 0; base < own; base += gpb) {
      const int l = base + grp;
      const bool live = l < own;
      const int64_t p = cp(l);
      float G[D * D] = {};
      if (live) {
        const float4 va = T.V[l];
        const float vav[3] = {va.x, va.y, va.z};
        const int nc = C.count(p);
#pragma unroll 2
        for (int t = lane; t < nc; t += L) {
          const int pk = C.slot(p, t);
          const float4 g = C.grad(p, t);
          const float gv[3] = {g.x, g.y, g.z};
          const float4 vb = cl.map_shared_rank(T.V, (unsigned)(pk >> 16))[pk & 0xffff];
          const float dv[3] = {vb.x - vav[0], vb.y - vav[1], vb.z - vav[2]};
          for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) G[i * d + j] = fmaf(dv[i], gv[j], G[i * d + j]);
        }
      }
      for (int o = L >> 1; o > 0; o >>= 1)
        for (int k = 0; k < d * d; ++k) G[k] += __shfl_xor_sync(0xffffffffu, G[k], o);
      if (live && lane == 0) {
        float B[D * D], dF[D * D], F[D * D];
#pragma unroll
        for (int k = 0; k < d * d; ++k) B[k] = C.b0(p, k);
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) {
            float s = 0.f;
            for (int k = 0; k < d; ++k) s += G[i * d + k] * B[k * d + j];
            dF[i * d + j] = s;
          }
        for (int k = 0; k < d * d; ++k) {
          T.dF[k * P + l] = dF[k];
          F[k] = T.F[k * P + l] + hh * dF[k];
        }
        if (more) solid_first_half<D, CS>(I, M, C, p, T, P, l, F, dF, hh);
        else
          for (int k = 0; k < d * d; ++k) T.F[k * P + l] = F[k];
      }
    }
    cl.sync();                             // P B0 published; every read of v done
  }
  // the owned particles back to global memory, with the step averages v~ and a~, and (single
  // time stepping) the next fluid step's cap
  const float inv = 1.0f / (float)kappa;
  vm = 0.f;
  am = 0.f;
  for (int l = threadIdx.x; l < own; l += blockDim.x) {
    const int64_t a = first + l;
    const float4 v = T.V[l], ac = T.acc[l], vs = T.vsum[l], as = T.asum[l];
    S.V[a] = v;
    S.X[a] = T.X[l];
    S.acc[a] = ac;
    S.vbar[a] = make_float4(vs.x * inv, vs.y * inv, vs.z * inv, 0.f);
    S.abar[a] = make_float4(as.x * inv, as.y * inv, as.z * inv, 0.f);
    for (int k = 0; k < d * d; ++k) {
      S.F[(int64_t)k * S.ns + a] = T.F[k * P + l];
      S.dFdt[(int64_t)k * S.ns + a] = T.dF[k * P + l];
    }
    vm = fmaxf(vm, v.x * v.x + v.y * v.y + v.z * v.z);
    am = fmaxf(am, ac.x * ac.x + ac.y * ac.y + ac.z * ac.z);
  }
  if (M.single_step && S.dt_cap) {
    // single time stepping: the next fluid step takes the solid's step from the state it
    // starts from (the same dt_S the next call computes first), a hair below it so kappa = 1
    cluster_vmax(cl, vm, am, red, blk);
    if (threadIdx.x == 0 && rank == 0) S.dt_cap[0] = solid_dt(M, vm, am) * (1.0 - 1e-9);
  }
}

// The solid's state in the caller's order (perm: internal index -> caller's), FP64.
__global__ void k_solid_export(int64_t ns, int d, const int* __restrict__ perm, const int4* __restrict__ X,
                               const float4* __restrict__ V, const float4* __restrict__ force,
                               const float* __restrict__ F, double lo0, double lo1, double lo2, double dq,
                               double* pos, double* vel, double* frc, double* Fout) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  const int64_t a = perm[i];               // the caller's index of internal particle i
  const int4 q = X[i];
  const int qv[3] = {q.x, q.y, q.z};
  const double lo[3] = {lo0, lo1, lo2};
  const float4 v = V[i], f = force[i];
  const float vv[3] = {v.x, v.y, v.z}, ff[3] = {f.x, f.y, f.z};
  for (int k = 0; k < d; ++k) {
    if (pos) pos[a * d + k] = lo[k] + (double)qv[k] * dq;
    if (vel) vel[a * d + k] = vv[k];
    if (frc) frc[a * d + k] = ff[k];
  }
  if (Fout)                                // F = I + H
    for (int k = 0; k < d * d; ++k) Fout[a * d * d + k] = (double)F[(int64_t)k * ns + i] + (k % (d + 1) == 0 ? 1.0 : 0.0);
}

}  // namespace
}  // namespace sph

// ---------------------------------------------------------------- the solid object ------
struct sph_solid {
  sph_handle* h = nullptr;
  std::string err;
  int64_t ns = 0;
  int dim = 2, cap = 0;
  int cluster = 1, threads = 32, lanes = 1, per_block = 1, tile_bytes = 0, row = 1;   // shape of the solid-step launch
  bool staged = false;          // constant rows staged in shared memory
  sph::SolidMat mat{};
  std::vector<void*> allocs;
  int4* X = nullptr;
  float4 *V = nullptr, *N = nullptr, *force = nullptr, *acc = nullptr, *vbar = nullptr, *abar = nullptr;
  float4 *gV = nullptr, *cA = nullptr;
  uint8_t* fixed = nullptr;
  float *F = nullptr, *dFdt = nullptr, *B0 = nullptr;   // F holds H = F - I
  float* vol = nullptr;         // reference volumes
  int *nb = nullptr, *cnt = nullptr, *near = nullptr, *box = nullptr, *dev_err = nullptr, *kappa_last = nullptr;
  int* n_near = nullptr;        // length of the near-fluid list (device)
  long long* steps = nullptr;
  int* perm = nullptr;          // internal index -> the caller's (device)
  int4 *sbox = nullptr, *fbox = nullptr;   // chunk boxes: solid, near fluid list
  std::vector<int> perm_host;
  uint32_t *flag = nullptr, *off = nullptr, *scan_tmp = nullptr;
};

namespace {

int sfail(sph_solid* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

template <typename T>
bool salloc(sph_solid* s, T** p, size_t count) {
  *p = nullptr;
  if (cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  s->allocs.push_back((void*)*p);
  return true;
}

sph::SolidPtrs ptrs(sph_solid* s) {
  sph::SolidPtrs P{};
  P.ns = s->ns;
  P.X = s->X;
  P.V = s->V;
  P.fixed = s->fixed;
  P.vol = s->vol;
  P.F = s->F;
  P.dFdt = s->dFdt;
  P.B0 = s->B0;
  P.nb = s->nb;
  P.cnt = s->cnt;
  P.gV = s->gV;
  P.cA = s->cA;
  P.force = s->force;
  P.acc = s->acc;
  P.vbar = s->vbar;
  P.abar = s->abar;
  P.steps = s->steps;
  P.kappa_last = s->kappa_last;
  P.dt_cap = s->h ? s->h->b.dt_cap : nullptr;
  P.g = s->h ? s->h->b.glob : nullptr;
  P.lanes = s->lanes;
  P.per_block = s->per_block;
  P.row = s->row;
  return P;
}

const void* solid_kernel(int dim, bool staged) {
  if (dim == 2) return staged ? (const void*)sph::k_solid_steps<2, true> : (const void*)sph::k_solid_steps<2, false>;
  return staged ? (const void*)sph::k_solid_steps<3, true> : (const void*)sph::k_solid_steps<3, false>;
}

// Shape of the solid-step launch: `lanes` per particle from the longest reference row (about
// six neighbours a lane); a cluster of c blocks, each holding ceil(ns / c) particles in its
// shared memory, with the constant rows too where they fit. c aims at eight or more busy
// warps a block, and stays within what the device schedules (16 blocks where non-portable
// cluster sizes are allowed) and within each block's shared memory. Returns false when no
// cluster holds the solid.
bool choose_cluster(sph_solid* s, int max_row) {
  int L = 1;
  while (L < 32 && L * 6 < max_row) L <<= 1;
  s->lanes = L;
  s->row = std::max(max_row, 1);
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int budget = optin - 1024;         // the kernel's static shared memory and a margin
  for (int cs = 1; cs >= 0; --cs) {        // constants staged in shared memory where they fit
    const void* kern = solid_kernel(s->dim, cs != 0);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, budget) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    auto bytes_for = [&](int P) {
      return (int64_t)sph::solid_tile_bytes(s->dim, P) + (cs ? (int64_t)P * sph::solid_const_bytes(s->dim, s->row) : 0);
    };
    const int64_t per = bytes_for(1) + 16;
    const int64_t c_mem = (s->ns + budget / per - 1) / std::max<int64_t>(budget / per, 1);
    const int64_t c_busy = (s->ns * L + 255) / 256;
    const int c0 = (int)std::max<int64_t>(c_mem, std::min<int64_t>(16, c_busy));
    std::vector<int> order;
    for (int c = c0; c >= (int)std::max<int64_t>(c_mem, 1); --c) order.push_back(c);
    for (int c = c0 + 1; c <= 16; ++c) order.push_back(c);
    for (int c : order) {
      const int P = (int)((s->ns + c - 1) / c);
      const int64_t bytes = bytes_for(P);
      if (bytes > budget) continue;
      // threads: the owned particles' lane groups, whole warps, at most one block's limit
      const int threads = (int)std::min<int64_t>(sph::kSolidThreads, std::max<int64_t>(32, ((int64_t)P * L + 31) / 32 * 32));
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      cfg.gridDim = dim3((unsigned)c);
      cfg.blockDim = dim3((unsigned)threads);
      cfg.dynamicSmemBytes = (size_t)bytes;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)c;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int active = 0;
      if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0) {
        s->cluster = c;
        s->threads = threads;
        s->per_block = P;
        s->tile_bytes = (int)bytes;
        s->staged = cs != 0;
        return true;
      }
      cudaGetLastError();
    }
  }
  return false;
}

void cluster_config(const sph_solid* s, cudaStream_t st, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3((unsigned)s->cluster);
  cfg->blockDim = dim3((unsigned)s->threads);
  cfg->dynamicSmemBytes = (size_t)s->tile_bytes;
  cfg->stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)s->cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg->attrs = at;
  cfg->numAttrs = 1;
}

}  // namespace

// Hooks called by the fluid's loop (sph_api.cu) when a solid is attached.
void sph_fsi_after_build(sph_handle* h, cudaStream_t st, int64_t* launches) {
  sph_solid* s = h->solid;
  if (!s || s->ns == 0) return;
  const sph::Buffers& b = h->b;
  const sph::Inst& I = b.inst0;
  const int pad = (int)std::min<double>(3.0 * I.h_d / I.dq_d, 1e9);
  sph::k_solid_bbox<<<1, sph::kSolidThreads, 0, st>>>(s->ns, s->X, pad, s->box);
  if (b.n > 0) {
    sph::k_near_flags<<<sph::fgrid(b.n), sph::kFBlock, 0, st>>>(b.n, b.dim, b.PS, s->box, s->flag);
    int64_t dummy = 0;
    sph::scan_exclusive(s->flag, s->off, b.n, s->scan_tmp, st, &dummy);
    sph::k_near_compact<<<sph::fgrid(b.n), sph::kFBlock, 0, st>>>(b.n, s->flag, s->off, s->near, s->n_near);
    *launches += 3 + dummy;
  }
  *launches += 1;
}

void sph_fsi_set_gravity(sph_handle* h, const double* g) {
  sph_solid* s = h->solid;
  if (!s) return;
  for (int a = 0; a < 3; ++a) s->mat.g[a] = a < s->dim ? (float)g[a] : 0.f;
}

void sph_fsi_after_pressure(sph_handle* h, cudaStream_t st, int64_t* launches) {
  sph_solid* s = h->solid;
  if (!s || s->ns == 0 || h->b.n == 0) return;
  sph::Buffers& b = h->b;
  // chunk boxes of the solid's positions and of the near fluid list's mid-point positions;
  // then a warp per near fluid particle (the list's length is on the device), a warp per
  // solid particle
  sph::k_chunk_boxes<<<sph::wgrid((s->ns + 31) / 32), sph::kFBlock, 0, st>>>(s->ns, nullptr, nullptr, s->X, s->sbox);
  sph::k_chunk_boxes<<<sph::wgrid((b.n + 31) / 32), sph::kFBlock, 0, st>>>(0, s->n_near, s->near, b.PH, s->fbox);
  auto fp = b.dim == 2 ? sph::k_fsi_fluid_pressure<2> : sph::k_fsi_fluid_pressure<3>;
  fp<<<sph::wgrid(b.n), sph::kFBlock, 0, st>>>(b.inst0, s->n_near, s->near, b.PH, b.VH, b.VS, b.mass, b.ctrl, s->ns,
                                               s->X, s->N, s->vbar, s->abar, s->sbox, b.acc_keep);
  auto sf = b.dim == 2 ? sph::k_fsi_solid_force<2> : sph::k_fsi_solid_force<3>;
  sf<<<sph::wgrid(s->ns), sph::kFBlock, 0, st>>>(b.inst0, s->n_near, s->near, b.PH, b.VS, b.mass, b.ctrl, s->ns, s->X,
                                                 s->N, s->vbar, s->abar, s->fbox, s->force);
  sph::Buffers vb = b;                     // |v|max over the corrected new velocities
  vb.VS = b.VH;
  sph::launch_vmax(vb, st, launches);
  *launches += 4;
}

void sph_fsi_after_density(sph_handle* h, cudaStream_t st, int64_t* launches) {
  sph_solid* s = h->solid;
  if (!s || s->ns == 0) return;
  sph::Buffers& b = h->b;
  if (b.n > 0) {
    auto fc = b.dim == 2 ? sph::k_fsi_fluid_continuity<2> : sph::k_fsi_fluid_continuity<3>;
    fc<<<sph::wgrid(b.n), sph::kFBlock, 0, st>>>(b.inst0, s->n_near, s->near, b.PS, b.VS, b.PH, b.ctrl, s->ns, s->X,
                                                 s->N, s->vbar, s->abar, s->sbox);
    *launches += 1;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cluster_config(s, st, &cfg, at);
  auto ks = b.dim == 2 ? (s->staged ? sph::k_solid_steps<2, true> : sph::k_solid_steps<2, false>)
                       : (s->staged ? sph::k_solid_steps<3, true> : sph::k_solid_steps<3, false>);
  cudaLaunchKernelEx(&cfg, ks, b.inst0, s->mat, ptrs(s), (const sph::Ctrl*)b.ctrl);
  *launches += 1;
}

extern "C" {

int sph_solid_create(sph_handle* h, const sph_solid_params* p, int64_t n, const double* pos, const double* vol,
                     const double* normal, const int32_t* fixed, sph_solid** out) {
  if (!out) return SPH_E_INVALID;
  *out = nullptr;
  if (!h || !p) return SPH_E_INVALID;
  sph_solid* s = new sph_solid();
  *out = s;
  if (h->solid) return sfail(s, SPH_E_INVALID, "the handle already has a solid");
  if (h->b.n_inst != 1) return sfail(s, SPH_E_INVALID, "a solid needs a single-tank handle");
  if (n < 1 || n > sph::kMaxSolid) return sfail(s, SPH_E_INVALID, "solid particle count must be in [1, 16384]");
  if (!pos || !vol || !normal) return sfail(s, SPH_E_INVALID, "pos, vol and normal are required");
  if (p->model != SPH_SOLID_LINEAR && p->model != SPH_SOLID_NEO_HOOKEAN) return sfail(s, SPH_E_INVALID, "unknown model");
  if (!(p->rho0 > 0.0 && p->youngs > 0.0 && p->poisson > -1.0 && p->poisson < 0.5 && p->h > 0.0) ||
      !std::isfinite(p->rho0 + p->youngs + p->poisson + p->h))
    return sfail(s, SPH_E_INVALID, "need rho0, youngs, h > 0 and -1 < poisson < 0.5");
  const int d = h->b.dim;
  s->h = h;
  s->ns = n;
  s->dim = d;
  // host copies of the caller's arrays (host or device memory)
  std::vector<double> hp((size_t)n * d), hv((size_t)n), hn((size_t)n * d);
  std::vector<int32_t> hf((size_t)n, 0);
  if (cudaMemcpy(hp.data(), pos, sizeof(double) * n * d, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(hv.data(), vol, sizeof(double) * n, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(hn.data(), normal, sizeof(double) * n * d, cudaMemcpyDefault) != cudaSuccess ||
      (fixed && cudaMemcpy(hf.data(), fixed, sizeof(int32_t) * n, cudaMemcpyDefault) != cudaSuccess)) {
    cudaGetLastError();
    return sfail(s, SPH_E_CUDA, "copy of the solid's arrays failed");
  }
  // Internal order: the particles sorted along a Morton curve of their reference positions
  // (cells of the lattice spacing), so that each block of the solid-step cluster owns a
  // compact patch and most reference neighbours share its shared memory. perm maps an
  // internal index to the caller's.
  {
    const double dps = std::pow(hv[0], 1.0 / d);
    if (!(dps > 0.0) || !std::isfinite(dps)) return sfail(s, SPH_E_INVALID, "solid volumes must be positive");
    double lo[3] = {1e300, 1e300, 1e300};
    for (int64_t a = 0; a < n; ++a)
      for (int k = 0; k < d; ++k) lo[k] = std::min(lo[k], hp[a * d + k]);
    std::vector<uint64_t> key((size_t)n);
    for (int64_t a = 0; a < n; ++a) {
      uint64_t m = 0;
      for (int k = 0; k < d; ++k) {
        const double c = std::floor((hp[a * d + k] - lo[k]) / dps);
        const uint64_t ci = (uint64_t)std::min(65535.0, std::max(0.0, c));
        for (int bit = 0; bit < 16; ++bit) m |= ((ci >> bit) & 1u) << (bit * d + k);
      }
      key[(size_t)a] = m;
    }
    s->perm_host.resize((size_t)n);
    for (int64_t a = 0; a < n; ++a) s->perm_host[(size_t)a] = (int)a;
    std::stable_sort(s->perm_host.begin(), s->perm_host.end(), [&](int x, int y) { return key[x] < key[y]; });
    std::vector<double> p2((size_t)n * d), v2((size_t)n), n2((size_t)n * d);
    std::vector<int32_t> f2((size_t)n);
    for (int64_t k2 = 0; k2 < n; ++k2) {
      const int64_t a = s->perm_host[(size_t)k2];
      for (int k = 0; k < d; ++k) {
        p2[k2 * d + k] = hp[a * d + k];
        n2[k2 * d + k] = hn[a * d + k];
      }
      v2[k2] = hv[a];
      f2[k2] = hf[a];
    }
    hp.swap(p2);
    hv.swap(v2);
    hn.swap(n2);
    hf.swap(f2);
  }
  const double nu = p->poisson, E = p->youngs;
  s->mat.model = p->model;
  s->mat.dim = d;
  s->mat.single_step = p->single_step ? 1 : 0;
  s->mat.mu = (float)(E / (2.0 * (1.0 + nu)));
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  s->mat.lam = (float)lam;
  s->mat.rho0 = (float)p->rho0;
  s->mat.h = p->h;
  s->mat.c = std::sqrt((lam + 2.0 * (E / (2.0 * (1.0 + nu))) / 3.0) / p->rho0);
  for (int a = 0; a < 3; ++a) s->mat.g[a] = a < d ? (float)h->params[0].gravity[a] : 0.f;
  // capacity of the reference rows: the lattice count within 2h plus margin
  const double dpr = std::pow(hv[0], 1.0 / d);
  const double rr = 2.0 * p->h / dpr;
  s->cap = (int)std::ceil((d == 2 ? 3.2 * rr * rr : 4.3 * rr * rr * rr)) + 8;
  const sph::Inst& I = h->b.inst0;
  std::vector<int4> hX((size_t)n);
  std::vector<float4> hN((size_t)n);
  std::vector<uint8_t> hfx((size_t)n);
  std::vector<float> hvol((size_t)n);
  for (int64_t a = 0; a < n; ++a) {
    int q[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
      const double v = (hp[a * d + k] - I.lo[k]) / I.dq_d;
      if (!(v > 0.0 && v < 2147483000.0)) return sfail(s, SPH_E_DOMAIN, "a solid particle lies outside the cell grid");
      q[k] = (int)std::llrint(v);
    }
    float vb = (float)hv[a];
    hvol[a] = vb;
    int vbits;
    std::memcpy(&vbits, &vb, sizeof(int));
    hX[a] = make_int4(q[0], q[1], q[2], vbits);
    hN[a] = make_float4((float)hn[a * d], (float)hn[a * d + 1], d == 3 ? (float)hn[a * d + 2] : 0.f, 0.f);
    hfx[a] = hf[a] ? 1 : 0;
  }
  const size_t dd = (size_t)d * d;
  bool ok = salloc(s, &s->X, n) && salloc(s, &s->V, n) && salloc(s, &s->N, n) && salloc(s, &s->force, n) &&
            salloc(s, &s->acc, n) && salloc(s, &s->vbar, n) && salloc(s, &s->abar, n) &&
            salloc(s, &s->fixed, n) && salloc(s, &s->vol, n) && salloc(s, &s->F, dd * n) &&
            salloc(s, &s->dFdt, dd * n) && salloc(s, &s->B0, dd * n) &&
            salloc(s, &s->nb, (size_t)s->cap * n) && salloc(s, &s->cnt, n) && salloc(s, &s->gV, (size_t)s->cap * n) && salloc(s, &s->cA, n) &&
            salloc(s, &s->box, 6) && salloc(s, &s->dev_err, 1) && salloc(s, &s->kappa_last, 1) &&
            salloc(s, &s->n_near, 1) &&
            salloc(s, &s->steps, 1) && salloc(s, &s->perm, n) && salloc(s, &s->sbox, 2 * ((n + 31) / 32)) &&
            salloc(s, &s->fbox, 2 * ((std::max<int64_t>(h->b.n, 1) + 31) / 32)) && salloc(s, &s->near, std::max<int64_t>(h->b.n, 1)) &&
            salloc(s, &s->flag, std::max<int64_t>(h->b.n, 1)) && salloc(s, &s->off, std::max<int64_t>(h->b.n, 1) + 1) &&
            salloc(s, &s->scan_tmp, sph::scan_tmp_elems(std::max<int64_t>(h->b.n, 1)));
  if (!ok) return sfail(s, SPH_E_OOM, "device allocation of the solid failed");
  double *dx0 = nullptr, *dvol = nullptr;
  if (!salloc(s, &dx0, (size_t)n * d) || !salloc(s, &dvol, n)) return sfail(s, SPH_E_OOM, "device allocation failed");
  if (cudaMemcpy(s->X, hX.data(), sizeof(int4) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->N, hN.data(), sizeof(float4) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->fixed, hfx.data(), n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->perm, s->perm_host.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->vol, hvol.data(), sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->F, 0, sizeof(float) * dd * n) != cudaSuccess ||          // H = F - I = 0
      cudaMemcpy(dx0, hp.data(), sizeof(double) * n * d, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dvol, hv.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->dFdt, 0, sizeof(float) * dd * n) != cudaSuccess ||
      cudaMemset(s->V, 0, sizeof(float4) * n) != cudaSuccess || cudaMemset(s->force, 0, sizeof(float4) * n) != cudaSuccess ||
      cudaMemset(s->acc, 0, sizeof(float4) * n) != cudaSuccess || cudaMemset(s->vbar, 0, sizeof(float4) * n) != cudaSuccess ||
      cudaMemset(s->abar, 0, sizeof(float4) * n) != cudaSuccess || cudaMemset(s->dev_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(s->steps, 0, sizeof(long long)) != cudaSuccess ||
      cudaMemset(s->n_near, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, SPH_E_CUDA, "initialising the solid failed");
  }
  sph::k_solid_setup<<<sph::fgrid(n), sph::kFBlock>>>(n, d, p->h, dx0, dvol, s->cap, s->nb, s->cnt, s->gV, s->cA, s->B0,
                                                      s->dev_err);
  int derr = 0;
  if (cudaMemcpy(&derr, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, SPH_E_CUDA, "solid set-up failed");
  }
  if (derr & 1) return sfail(s, SPH_E_CAPACITY, "a solid particle has more reference neighbours than the capacity");
  if (derr & 2) return sfail(s, SPH_E_INVALID, "a solid particle's correction matrix is singular (too few neighbours)");
  std::vector<int> hcnt((size_t)n);
  if (cudaMemcpy(hcnt.data(), s->cnt, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, SPH_E_CUDA, "solid set-up failed");
  }
  if (!choose_cluster(s, *std::max_element(hcnt.begin(), hcnt.end())))
    return sfail(s, SPH_E_CAPACITY, "the solid does not fit the shared memory of one thread-block cluster");
  sph::k_solid_pack_rows<<<sph::fgrid(n), sph::kFBlock>>>(n, s->cap, s->cnt, s->per_block, s->nb);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, SPH_E_CUDA, "solid set-up failed");
  }
  if (p->single_step) {
    double* cap = nullptr;
    if (!salloc(s, &cap, 1) || cudaMemset(cap, 0, sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return sfail(s, SPH_E_OOM, "device allocation of the step cap failed");
    }
    h->b.dt_cap = cap;
  }
  h->solid = s;
  sph_drop_graph(h);                       // the loop now includes the coupling kernels
  h->cells_valid = false;                  // the near list comes with the next configuration update
  return SPH_OK;
}

void sph_solid_destroy(sph_solid* s) {
  if (!s) return;
  if (s->h && s->h->solid == s) {
    s->h->solid = nullptr;
    s->h->b.dt_cap = nullptr;              // freed with the solid's allocations below
    sph_drop_graph(s->h);
  }
  for (void* p : s->allocs) cudaFree(p);
  delete s;
}

const char* sph_solid_last_error(const sph_solid* s) { return s ? s->err.c_str() : "null solid"; }

int64_t sph_solid_size(const sph_solid* s) { return s ? s->ns : -1; }

int sph_solid_get_state(sph_handle* h, sph_solid* s, double* pos, double* vel, double* force, double* F,
                        int64_t* solid_steps, void* stream) {
  if (!h || !s || s->h != h) return SPH_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const int d = s->dim;
  const size_t n = (size_t)s->ns;
  double* dst[4] = {pos, vel, force, F};
  const size_t sz[4] = {n * d, n * d, n * d, n * d * d};
  double* tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(double) * (3 * n * d + n * d * d)) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, SPH_E_OOM, "staging allocation failed");
  }
  double* t[4] = {tmp, tmp + n * d, tmp + 2 * n * d, tmp + 3 * n * d};
  const sph::Inst& I = h->b.inst0;
  sph::k_solid_export<<<sph::fgrid(s->ns), sph::kFBlock, 0, st>>>(s->ns, d, s->perm, s->X, s->V, s->force, s->F, I.lo[0],
                                                                  I.lo[1], I.lo[2], I.dq_d, t[0], t[1], t[2], t[3]);
  int rc = SPH_OK;
  for (int k = 0; k < 4; ++k)
    if (dst[k] && cudaMemcpyAsync(dst[k], t[k], sizeof(double) * sz[k], cudaMemcpyDefault, st) != cudaSuccess)
      rc = SPH_E_CUDA;
  long long steps = 0;
  if (cudaMemcpyAsync(&steps, s->steps, sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SPH_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = SPH_E_CUDA;
  cudaFree(tmp);
  if (rc != SPH_OK) {
    cudaGetLastError();
    return sfail(s, rc, "copy of the solid's state failed");
  }
  if (solid_steps) *solid_steps = steps;
  return SPH_OK;
}

}  // extern "C"
