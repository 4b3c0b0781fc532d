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
//    the fluid force held, in one single-block kernel; v~ and a~ become their averages.
// The fluid particles near the solid (inside its bounding box widened by 3 h_F) are listed
// once per configuration update, in storage order.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_handle.h"
#include "sph_kernels.h"

namespace sph {
namespace {

constexpr int kFBlock = 128;
constexpr int kSolidThreads = 1024;       // the solid steps run in one block
constexpr int kMaxSolid = 16 * kSolidThreads;

inline unsigned fgrid(int64_t n) { return (unsigned)((n + kFBlock - 1) / kFBlock); }

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
// One thread per solid particle: its neighbours within 2 h_S in the reference configuration
// (ascending index), their kernel gradients, and B0 (FP64, then stored in FP32).
__global__ void k_solid_setup(int64_t ns, int d, double h, const double* __restrict__ x0,
                              const double* __restrict__ vol, int cap, int* __restrict__ nb,
                              int* __restrict__ cnt, float4* __restrict__ gW, float* __restrict__ B0, int* err) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  const double pi = 3.14159265358979323846;
  const double alpha = d == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
  double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
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
    gW[(int64_t)c * ns + a] = make_float4((float)g[0], (float)g[1], (float)g[2], 0.f);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) M[i * d + j] += vol[b] * (-r[i]) * g[j];   // (r0_b - r0_a) (x) grad
    ++c;
  }
  cnt[a] = c;
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

template <int D>
__global__ void __launch_bounds__(kFBlock)
k_fsi_fluid_pressure(const Inst I, const int* __restrict__ n_near_p, const int* __restrict__ near, const int4* __restrict__ PH,
                     float4* __restrict__ VH, const float4* __restrict__ VS, const float* __restrict__ mass,
                     const Ctrl* __restrict__ ctrl, int64_t ns, const int4* __restrict__ X,
                     const float4* __restrict__ N, const float4* __restrict__ vbar, const float4* __restrict__ abar,
                     float4* __restrict__ acc_keep) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *n_near_p) return;
  const double dtd = ctrl[0].dt;
  if (dtd == 0.0) return;
  const int i = near[k];
  const int4 qi = PH[i];
  const float dev_i = i2f(qi.w);
  const float m_i = mass ? mass[i] : I.mass;
  const float4 vi = VS[i];
  float s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
  for (int64_t a = 0; a < ns; ++a) {
    const int4 qa = X[a];
    const FsiPair P = fsi_geometry<D>(qi, qa, I);
    if (!P.in) continue;
    const float3 f = fsi_force(P, dev_i, m_i, vi, i2f(qa.w), N[a], vbar[a], abar[a], I);
    kahan_add(s[0], c[0], f.x / m_i);
    kahan_add(s[1], c[1], f.y / m_i);
    if (D == 3) kahan_add(s[2], c[2], f.z / m_i);
  }
  const float dt = (float)dtd;
  const float ax = s[0] - c[0], ay = s[1] - c[1], az = s[2] - c[2];
  float4 v = VH[i];
  v.x += dt * ax;
  v.y += dt * ay;
  if (D == 3) v.z += dt * az;
  VH[i] = v;
  if (acc_keep) {
    float4 a = acc_keep[i];
    a.x += ax;
    a.y += ay;
    a.z += az;
    acc_keep[i] = a;
  }
}

template <int D>
__global__ void __launch_bounds__(kFBlock)
k_fsi_solid_force(const Inst I, const int* __restrict__ n_near_p, const int* __restrict__ near, const int4* __restrict__ PH,
                  const float4* __restrict__ VS, const float* __restrict__ mass, const Ctrl* __restrict__ ctrl,
                  int64_t ns, const int4* __restrict__ X, const float4* __restrict__ N,
                  const float4* __restrict__ vbar, const float4* __restrict__ abar, float4* __restrict__ force) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  if (ctrl[0].dt == 0.0) return;
  const int4 qa = X[a];
  const float V_a = i2f(qa.w);
  const float4 n = N[a], vb = vbar[a], ab = abar[a];
  const int n_near = *n_near_p;
  float s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
  for (int k = 0; k < n_near; ++k) {
    const int i = near[k];
    const int4 qi = PH[i];
    const FsiPair P = fsi_geometry<D>(qi, qa, I);
    if (!P.in) continue;
    const float m_i = mass ? mass[i] : I.mass;
    const float3 f = fsi_force(P, i2f(qi.w), m_i, VS[i], V_a, n, vb, ab, I);
    kahan_add(s[0], c[0], -f.x);
    kahan_add(s[1], c[1], -f.y);
    if (D == 3) kahan_add(s[2], c[2], -f.z);
  }
  force[a] = make_float4(s[0] - c[0], s[1] - c[1], s[2] - c[2], 0.f);
}

template <int D>
__global__ void __launch_bounds__(kFBlock)
k_fsi_fluid_continuity(const Inst I, const int* __restrict__ n_near_p, const int* __restrict__ near, int4* __restrict__ PS,
                       float4* __restrict__ VS, const int4* __restrict__ PH, const Ctrl* __restrict__ ctrl,
                       int64_t ns, const int4* __restrict__ X, const float4* __restrict__ N,
                       const float4* __restrict__ vbar, const float4* __restrict__ abar) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *n_near_p) return;
  const double dtd = ctrl[0].dt;
  if (dtd == 0.0) return;
  const int i = near[k];
  int4 qi = PS[i];                         // r^{n+1}, and the new density deviation in w
  float4 vi = VS[i];                       // v^{n+1}
  const float dev_h = i2f(PH[i].w);        // rho_i is the mid-point density, as in the fluid pass
  const float rho_i = I.rho0 + dev_h;
  const float p_i = I.c0sq * dev_h;
  float s = 0.f, c = 0.f;
  for (int64_t a = 0; a < ns; ++a) {
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
    kahan_add(s, c, 2.0f * rho_i * i2f(qa.w) * (Us - UL) * P.dW);
  }
  const float drho = s - c;
  const float hdt = 0.5f * (float)dtd;
  qi.w = f2i(i2f(qi.w) + hdt * drho);
  vi.w += drho;
  PS[i] = qi;
  VS[i] = vi;
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
  float *F, *dFdt, *PB;   // F: the displacement gradient H = F - I
  const float* B0;
  const int* nb;
  const int* cnt;
  const float4* gW;
  const float4* force;
  float4 *acc, *vbar, *abar, *vsum, *asum;
  long long* steps;      // solid steps taken, total
  int* kappa_last;
  double* dt_cap;        // the fluid's cap (single time stepping), or NULL
};

// All kappa solid steps of one fluid acoustic step, one block, __syncthreads between the
// three phases of each step.
template <int D>
__global__ void __launch_bounds__(kSolidThreads)
k_solid_steps(const Inst I, SolidMat M, SolidPtrs S, const Ctrl* __restrict__ ctrl) {
  const double dtF = ctrl[0].dt;
  if (dtF == 0.0) return;
  constexpr int d = D;
  const int64_t ns = S.ns;
  // Eq. dts-advection from the solid's state at the start of the fluid step (R25)
  __shared__ float red_v[kSolidThreads / 32], red_a[kSolidThreads / 32];
  __shared__ int s_kappa;
  float vm = 0.f, am = 0.f;
  for (int64_t a = threadIdx.x; a < ns; a += blockDim.x) {
    const float4 v = S.V[a], ac = S.acc[a];
    vm = fmaxf(vm, v.x * v.x + v.y * v.y + v.z * v.z);
    am = fmaxf(am, ac.x * ac.x + ac.y * ac.y + ac.z * ac.z);
    S.vsum[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    S.asum[a] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) {
    vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red_v[threadIdx.x >> 5] = vm;
    red_a[threadIdx.x >> 5] = am;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      vm = fmaxf(vm, red_v[w]);
      am = fmaxf(am, red_a[w]);
    }
    double dts = M.h / (M.c + sqrt((double)vm));
    if (am > 0.f) dts = fmin(dts, sqrt(M.h / sqrt((double)am)));
    dts *= 0.6;
    s_kappa = (int)floor(dtF / dts) + 1;
    *S.kappa_last = s_kappa;
    *S.steps += s_kappa;
  }
  __syncthreads();
  const int kappa = s_kappa;
  const double hd = dtF / kappa;
  const float h = (float)hd, hh = 0.5f * h;
  for (int step = 0; step < kappa; ++step) {
    // phase 1: F to the mid point, r half a step, P B0
    for (int64_t a = threadIdx.x; a < ns; a += blockDim.x) {
      float F[D * D], dF[D * D], B[D * D], P[D * D], PB[D * D];
      load_mat<D>(S.F, ns, a, F);
      load_mat<D>(S.dFdt, ns, a, dF);
      for (int k = 0; k < d * d; ++k) F[k] += hh * dF[k];
      store_mat<D>(S.F, ns, a, F);
      if (!S.fixed[a]) {
        const float4 v = S.V[a];
        int4 q = S.X[a];
        q.x += __float2int_rn(hh * v.x * I.inv_dq);
        q.y += __float2int_rn(hh * v.y * I.inv_dq);
        if (d == 3) q.z += __float2int_rn(hh * v.z * I.inv_dq);
        S.X[a] = q;
      }
      first_piola<D>(M, F, P);
      load_mat<D>(S.B0, ns, a, B);
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          float s = 0.f;
          for (int k = 0; k < d; ++k) s += P[i * d + k] * B[k * d + j];
          PB[i * d + j] = s;
        }
      store_mat<D>(S.PB, ns, a, PB);
    }
    __syncthreads();
    // phase 2: dv/dt, v, r the second half
    for (int64_t a = threadIdx.x; a < ns; a += blockDim.x) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!S.fixed[a]) {
        const float Va = i2f(S.X[a].w);
        const float ma = M.rho0 * Va;
        float PBa[D * D];
        load_mat<D>(S.PB, ns, a, PBa);
        float s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
        const int nc = S.cnt[a];
        for (int t = 0; t < nc; ++t) {
          const int b = S.nb[(int64_t)t * ns + a];
          const float4 g = S.gW[(int64_t)t * ns + a];
          const float gv[3] = {g.x, g.y, g.z};
          const float w = Va * i2f(S.X[b].w);
          for (int i = 0; i < d; ++i) {
            float x = 0.f;
            for (int j = 0; j < d; ++j) x += 0.5f * (PBa[i * d + j] + S.PB[(int64_t)(i * d + j) * ns + b]) * gv[j];
            kahan_add(s[i], c[i], w * x);
          }
        }
        const float4 f = S.force[a];
        acc.x = 2.0f * (s[0] - c[0]) / ma + M.g[0] + f.x / ma;
        acc.y = 2.0f * (s[1] - c[1]) / ma + M.g[1] + f.y / ma;
        acc.z = d == 3 ? 2.0f * (s[2] - c[2]) / ma + M.g[2] + f.z / ma : 0.f;
        float4 v = S.V[a];
        v.x += h * acc.x;
        v.y += h * acc.y;
        v.z += h * acc.z;
        S.V[a] = v;
        int4 q = S.X[a];
        q.x += __float2int_rn(hh * v.x * I.inv_dq);
        q.y += __float2int_rn(hh * v.y * I.inv_dq);
        if (d == 3) q.z += __float2int_rn(hh * v.z * I.inv_dq);
        S.X[a] = q;
      }
      S.acc[a] = acc;
      const float4 v = S.V[a];
      float4 vs = S.vsum[a], as = S.asum[a];
      vs.x += v.x; vs.y += v.y; vs.z += v.z;
      as.x += acc.x; as.y += acc.y; as.z += acc.z;
      S.vsum[a] = vs;
      S.asum[a] = as;
    }
    __syncthreads();
    // phase 3: dF/dt from the new velocities, F the second half
    for (int64_t a = threadIdx.x; a < ns; a += blockDim.x) {
      const float4 va = S.V[a];
      const float vav[3] = {va.x, va.y, va.z};
      float G[D * D] = {};
      const int nc = S.cnt[a];
      for (int t = 0; t < nc; ++t) {
        const int b = S.nb[(int64_t)t * ns + a];
        const float4 g = S.gW[(int64_t)t * ns + a];
        const float gv[3] = {g.x, g.y, g.z};
        const float4 vb = S.V[b];
        const float vbv[3] = {vb.x, vb.y, vb.z};
        const float Vb = i2f(S.X[b].w);
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) G[i * d + j] += Vb * (vbv[i] - vav[i]) * gv[j];
      }
      float B[D * D], dF[D * D], F[D * D];
      load_mat<D>(S.B0, ns, a, B);
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          float s = 0.f;
          for (int k = 0; k < d; ++k) s += G[i * d + k] * B[k * d + j];
          dF[i * d + j] = s;
        }
      store_mat<D>(S.dFdt, ns, a, dF);
      load_mat<D>(S.F, ns, a, F);
      for (int k = 0; k < d * d; ++k) F[k] += hh * dF[k];
      store_mat<D>(S.F, ns, a, F);
    }
    __syncthreads();
  }
  const float inv = 1.0f / (float)kappa;
  for (int64_t a = threadIdx.x; a < ns; a += blockDim.x) {
    const float4 vs = S.vsum[a], as = S.asum[a];
    S.vbar[a] = make_float4(vs.x * inv, vs.y * inv, vs.z * inv, 0.f);
    S.abar[a] = make_float4(as.x * inv, as.y * inv, as.z * inv, 0.f);
  }
  if (M.single_step && S.dt_cap) {
    // single time stepping: the next fluid step takes the solid's step from the state it
    // starts from (the same dt_S the next call computes first), a hair below it so kappa = 1
    __syncthreads();
    vm = 0.f;
    am = 0.f;
    for (int64_t a = threadIdx.x; a < ns; a += blockDim.x) {
      const float4 v = S.V[a], ac = S.acc[a];
      vm = fmaxf(vm, v.x * v.x + v.y * v.y + v.z * v.z);
      am = fmaxf(am, ac.x * ac.x + ac.y * ac.y + ac.z * ac.z);
    }
    for (int o = 16; o > 0; o >>= 1) {
      vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
      am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red_v[threadIdx.x >> 5] = vm;
      red_a[threadIdx.x >> 5] = am;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        vm = fmaxf(vm, red_v[w]);
        am = fmaxf(am, red_a[w]);
      }
      double dts = M.h / (M.c + sqrt((double)vm));
      if (am > 0.f) dts = fmin(dts, sqrt(M.h / sqrt((double)am)));
      S.dt_cap[0] = 0.6 * dts * (1.0 - 1e-9);
    }
  }
}

__global__ void k_solid_export(int64_t ns, int d, const int4* __restrict__ X, const float4* __restrict__ V,
                               const float4* __restrict__ force, const float* __restrict__ F, double lo0,
                               double lo1, double lo2, double dq, double* pos, double* vel, double* frc,
                               double* Fout) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  const int4 q = X[a];
  const int qv[3] = {q.x, q.y, q.z};
  const double lo[3] = {lo0, lo1, lo2};
  const float4 v = V[a], f = force[a];
  const float vv[3] = {v.x, v.y, v.z}, ff[3] = {f.x, f.y, f.z};
  for (int k = 0; k < d; ++k) {
    if (pos) pos[a * d + k] = lo[k] + (double)qv[k] * dq;
    if (vel) vel[a * d + k] = vv[k];
    if (frc) frc[a * d + k] = ff[k];
  }
  if (Fout)                                // F = I + H
    for (int k = 0; k < d * d; ++k) Fout[a * d * d + k] = (double)F[(int64_t)k * ns + a] + (k % (d + 1) == 0 ? 1.0 : 0.0);
}

}  // namespace
}  // namespace sph

// ---------------------------------------------------------------- the solid object ------
struct sph_solid {
  sph_handle* h = nullptr;
  std::string err;
  int64_t ns = 0;
  int dim = 2, cap = 0;
  sph::SolidMat mat{};
  std::vector<void*> allocs;
  int4* X = nullptr;
  float4 *V = nullptr, *N = nullptr, *force = nullptr, *acc = nullptr, *vbar = nullptr, *abar = nullptr;
  float4 *vsum = nullptr, *asum = nullptr, *gW = nullptr;
  uint8_t* fixed = nullptr;
  float *F = nullptr, *dFdt = nullptr, *PB = nullptr, *B0 = nullptr;   // F holds H = F - I
  int *nb = nullptr, *cnt = nullptr, *near = nullptr, *box = nullptr, *dev_err = nullptr, *kappa_last = nullptr;
  int* n_near = nullptr;        // length of the near-fluid list (device)
  long long* steps = nullptr;
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
  sph::SolidPtrs P;
  P.ns = s->ns;
  P.X = s->X;
  P.V = s->V;
  P.fixed = s->fixed;
  P.F = s->F;
  P.dFdt = s->dFdt;
  P.PB = s->PB;
  P.B0 = s->B0;
  P.nb = s->nb;
  P.cnt = s->cnt;
  P.gW = s->gW;
  P.force = s->force;
  P.acc = s->acc;
  P.vbar = s->vbar;
  P.abar = s->abar;
  P.vsum = s->vsum;
  P.asum = s->asum;
  P.steps = s->steps;
  P.kappa_last = s->kappa_last;
  P.dt_cap = s->h ? s->h->b.dt_cap : nullptr;
  return P;
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

void sph_fsi_after_pressure(sph_handle* h, cudaStream_t st, int64_t* launches) {
  sph_solid* s = h->solid;
  if (!s || s->ns == 0 || h->b.n == 0) return;
  sph::Buffers& b = h->b;
  // launched over every fluid slot: threads past the near list's length (on the device) exit
  auto fp = b.dim == 2 ? sph::k_fsi_fluid_pressure<2> : sph::k_fsi_fluid_pressure<3>;
  fp<<<sph::fgrid(b.n), sph::kFBlock, 0, st>>>(b.inst0, s->n_near, s->near, b.PH, b.VH, b.VS, b.mass, b.ctrl, s->ns,
                                               s->X, s->N, s->vbar, s->abar, b.acc_keep);
  auto sf = b.dim == 2 ? sph::k_fsi_solid_force<2> : sph::k_fsi_solid_force<3>;
  sf<<<sph::fgrid(s->ns), sph::kFBlock, 0, st>>>(b.inst0, s->n_near, s->near, b.PH, b.VS, b.mass, b.ctrl, s->ns, s->X,
                                                 s->N, s->vbar, s->abar, s->force);
  sph::Buffers vb = b;                     // |v|max over the corrected new velocities
  vb.VS = b.VH;
  sph::launch_vmax(vb, st, launches);
  *launches += 2;
}

void sph_fsi_after_density(sph_handle* h, cudaStream_t st, int64_t* launches) {
  sph_solid* s = h->solid;
  if (!s || s->ns == 0) return;
  sph::Buffers& b = h->b;
  if (b.n > 0) {
    auto fc = b.dim == 2 ? sph::k_fsi_fluid_continuity<2> : sph::k_fsi_fluid_continuity<3>;
    fc<<<sph::fgrid(b.n), sph::kFBlock, 0, st>>>(b.inst0, s->n_near, s->near, b.PS, b.VS, b.PH, b.ctrl, s->ns, s->X,
                                                 s->N, s->vbar, s->abar);
    *launches += 1;
  }
  auto ks = b.dim == 2 ? sph::k_solid_steps<2> : sph::k_solid_steps<3>;
  ks<<<1, sph::kSolidThreads, 0, st>>>(b.inst0, s->mat, ptrs(s), b.ctrl);
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
  for (int64_t a = 0; a < n; ++a) {
    int q[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
      const double v = (hp[a * d + k] - I.lo[k]) / I.dq_d;
      if (!(v > 0.0 && v < 2147483000.0)) return sfail(s, SPH_E_DOMAIN, "a solid particle lies outside the cell grid");
      q[k] = (int)std::llrint(v);
    }
    float vb = (float)hv[a];
    int vbits;
    std::memcpy(&vbits, &vb, sizeof(int));
    hX[a] = make_int4(q[0], q[1], q[2], vbits);
    hN[a] = make_float4((float)hn[a * d], (float)hn[a * d + 1], d == 3 ? (float)hn[a * d + 2] : 0.f, 0.f);
    hfx[a] = hf[a] ? 1 : 0;
  }
  const size_t dd = (size_t)d * d;
  bool ok = salloc(s, &s->X, n) && salloc(s, &s->V, n) && salloc(s, &s->N, n) && salloc(s, &s->force, n) &&
            salloc(s, &s->acc, n) && salloc(s, &s->vbar, n) && salloc(s, &s->abar, n) && salloc(s, &s->vsum, n) &&
            salloc(s, &s->asum, n) && salloc(s, &s->fixed, n) && salloc(s, &s->F, dd * n) &&
            salloc(s, &s->dFdt, dd * n) && salloc(s, &s->PB, dd * n) && salloc(s, &s->B0, dd * n) &&
            salloc(s, &s->nb, (size_t)s->cap * n) && salloc(s, &s->cnt, n) && salloc(s, &s->gW, (size_t)s->cap * n) &&
            salloc(s, &s->box, 6) && salloc(s, &s->dev_err, 1) && salloc(s, &s->kappa_last, 1) &&
            salloc(s, &s->n_near, 1) &&
            salloc(s, &s->steps, 1) && salloc(s, &s->near, std::max<int64_t>(h->b.n, 1)) &&
            salloc(s, &s->flag, std::max<int64_t>(h->b.n, 1)) && salloc(s, &s->off, std::max<int64_t>(h->b.n, 1) + 1) &&
            salloc(s, &s->scan_tmp, sph::scan_tmp_elems(std::max<int64_t>(h->b.n, 1)));
  if (!ok) return sfail(s, SPH_E_OOM, "device allocation of the solid failed");
  double *dx0 = nullptr, *dvol = nullptr;
  if (!salloc(s, &dx0, (size_t)n * d) || !salloc(s, &dvol, n)) return sfail(s, SPH_E_OOM, "device allocation failed");
  if (cudaMemcpy(s->X, hX.data(), sizeof(int4) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->N, hN.data(), sizeof(float4) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->fixed, hfx.data(), n, cudaMemcpyHostToDevice) != cudaSuccess ||
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
  sph::k_solid_setup<<<sph::fgrid(n), sph::kFBlock>>>(n, d, p->h, dx0, dvol, s->cap, s->nb, s->cnt, s->gW, s->B0,
                                                      s->dev_err);
  int derr = 0;
  if (cudaMemcpy(&derr, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, SPH_E_CUDA, "solid set-up failed");
  }
  if (derr & 1) return sfail(s, SPH_E_CAPACITY, "a solid particle has more reference neighbours than the capacity");
  if (derr & 2) return sfail(s, SPH_E_INVALID, "a solid particle's correction matrix is singular (too few neighbours)");
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
  sph::k_solid_export<<<sph::fgrid(s->ns), sph::kFBlock, 0, st>>>(s->ns, d, s->X, s->V, s->force, s->F, I.lo[0],
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
