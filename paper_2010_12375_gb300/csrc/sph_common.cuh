// Device-side data layout and per-pair physics of the WCSPH hot path.
//
// Particle state lives in HBM as two 16-byte records per fluid particle, in
// cell-sorted order:
//   P = int4  {qx, qy, qz, bits(rho - rho0)}   fixed-point position + density deviation
//   V = float4{vx, vy, vz, drho/dt}
// Positions are integers in units of dq (the cell size / 2^bits), so the high
// bits are the cell and the low bits the offset inside it; pair differences are
// exact integers and become floats exactly for |dq| < 2^24. Storing rho - rho0
// instead of rho keeps the pressure p = c0^2 (rho - rho0) (Eq. eqeos) free of
// cancellation.
// Wall particles (static) are
//   WP = int4  {qx, qy, qz, bits(V_w)}
//   WN = float4{nx, ny, nz, 0}                 unit normal into the fluid
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {

constexpr float kLimiter = 3.0f;        // dissipation limiter of the low-dissipation solver
constexpr double kLoopSlack = 1e-12;     // substep loop runs while tau < Dt_ad (1 - slack)
constexpr int kMaxSubstepsPerStep = 1000; // default bound of the device-side substep loop (normal: <= 6)

enum : int { ERR_DOMAIN = 1, ERR_NAN = 2, ERR_CAPACITY = 4, ERR_DT = 8, ERR_TIMEOUT = 16, ERR_BOUNDS = 32 };

// Per-instance constants (one tank), read-only on the device.
struct Inst {
  float h, inv_h, four_h2;       // h, 1/h, (2h)^2
  float dq;                      // position quantum (length units)
  float inv_dq;
  float c0, c0sq, rho0;
  float w_a;                     // alpha_d of the Wendland C2 kernel
  float dwr_a;                   // -5 alpha_d / h^2 : (dW/dr)/r = dwr_a (1 - q/2)^3
  float sig_hi, sig_lo;          // W(0) - sumW0 as a float pair (hi + lo)
  float rho0_over_sigma0;
  float kc;                      // limiter / c0 (low-dissipation solver)
  float qc0;                     // c0 / 4
  float hc0sq;                   // c0^2 / 2
  float inv_c0sq;                // 1 / c0^2
  float g[3];
  float eta;                     // rho0 * nu
  float mass;                    // uniform particle mass
  float p_tv;                    // background pressure p0 of the transport velocity (0 = off)
  int   ncell[3];                // cells per axis (position frame: q >> bits)
  int   scell[3];                // search cells per axis, 2 ncell (1 on an unused axis)
  int   period[3];               // period in quanta on periodic axes, else 0
  int   bits;
  int   sbits;                   // search cell of a particle: q >> sbits, sbits = bits - 1
  int   free_surface;
  int   max_sub;                 // bound of the substep loop of one advection step
  long long R2;                  // integer neighbour threshold
  long long cell_base;           // first global cell of this instance
  long long fluid_begin, fluid_end;
  long long wall_begin, wall_end;
  double h_d, c0_d, u_ref, nu, cfl_ad, cfl_ac;
  double lo[3];                  // cell-grid origin
  double dq_d;                   // position quantum in double precision
  double rho0_d;
};

// Per-instance time control (device, written by the 1-thread step kernels).
struct Ctrl {
  double t;          // simulated time
  double tau;        // time covered in the current advection step
  double dt_ad;      // current advection step
  double dt;         // current acoustic substep (0 = this instance is idle)
  unsigned int vmax2;// bits of max |v|^2 (non-negative floats order like unsigned ints)
  int done;          // current advection step covered
  long long substeps;
  long long adv_steps;
  int sub_in_step;   // substeps taken in the current advection step
  int pad;
};

// Device-wide status.
struct Global {
  int err;
  int active;              // some instance still needs substeps
  long long substeps;      // substep kernels executed (any instance active)
  long long bad_index;     // first particle that raised an error (diagnosis)
};

__device__ __forceinline__ float i2f(int v) { return __int_as_float(v); }
__device__ __forceinline__ int f2i(float v) { return __float_as_int(v); }

// Minimum-image integer difference on a periodic axis (period P quanta, 0 = none).
__device__ __forceinline__ int wrap_diff(int d, int P) {
  if (P) {
    int half = P >> 1;
    if (d > half) d -= P;
    else if (d < -half) d += P;
  }
  return d;
}

__device__ __forceinline__ int wrap_coord(int q, int P) {
  if (P) {
    if (q < 0) q += P;
    else if (q >= P) q -= P;
  }
  return q;
}

// Exact neighbour predicate on fixed-point positions: sum dq^2 < R2.
template <int D>
__device__ __forceinline__ bool within(const int4& a, const int4& b, const Inst& I) {
  int dx = wrap_diff(a.x - b.x, I.period[0]);
  int dy = wrap_diff(a.y - b.y, I.period[1]);
  long long d2 = (long long)dx * dx + (long long)dy * dy;
  if (D == 3) {
    int dz = wrap_diff(a.z - b.z, I.period[2]);
    d2 += (long long)dz * dz;
  }
  return d2 < I.R2;
}

// Kahan-compensated accumulation.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  float y = x - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Wendland C2 kernel value, support 2h.
__device__ __forceinline__ float kernel_W(float r, const Inst& I) {
  float q = r * I.inv_h;
  float t = fmaxf(1.0f - 0.5f * q, 0.0f);
  float t2 = t * t;
  return I.w_a * t2 * t2 * (1.0f + 2.0f * q);
}

// (dW/dr) / r of the Wendland C2 kernel: -5 alpha/h^2 (1 - q/2)^3, finite at r = 0.
__device__ __forceinline__ float kernel_dW_over_r(float r, const Inst& I) {
  float q = r * I.inv_h;
  float t = fmaxf(1.0f - 0.5f * q, 0.0f);
  return I.dwr_a * t * t * t;
}

}  // namespace sph

// ---- packed FP32 (two lanes per instruction) -------------------------------------------
// The relaxation kernels evaluate two neighbour pairs at a time in the .x/.y lanes
// of float2 values with sm_100+ packed FP32 instructions.
namespace sph {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // a - b, one rounding
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 max2(float2 a, float b) { return make_float2(fmaxf(a.x, b), fmaxf(a.y, b)); }
__device__ __forceinline__ float2 min2(float2 a, float b) { return make_float2(fminf(a.x, b), fminf(a.y, b)); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) {
  return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
}

// s += a*b with Kahan compensation kept negated in nc (the product is fused).
__device__ __forceinline__ void kahan2(float2& s, float2& nc, float2 a, float2 b) {
  float2 y = fma2(a, b, nc);
  float2 t = add2(s, y);
  nc = sub2(y, sub2(t, s));
  s = t;
}

// Exact int -> float of a fixed-point difference |d| < 2^22 with integer and FP32
// adds only: the bits of 1.5*2^23 + d, read as a float, minus 1.5*2^23. Larger |d|
// map to values of magnitude >= 2^22 quanta (>= 2h), which contribute nothing.
constexpr unsigned kMagicBits = 0x4B400000u;
constexpr float kMagic = 12582912.0f;

template <bool PER>
__device__ __forceinline__ float biased_diff(int qi, int qj, int period) {
  unsigned d;
  if (PER) d = (unsigned)wrap_diff(qi - qj, period) + kMagicBits;
  else d = (unsigned)qi - (unsigned)qj + kMagicBits;
  return __uint_as_float(d);
}

}  // namespace sph

// ---- neighbour table layout ---------------------------------------------------------------
// Slot s of particle i lives at int index ((s >> 2) * n + i) * 4 + (s & 3): quads of four
// slots are interleaved over particles, so a warp reads one quad row as 32 contiguous
// 16-byte loads. Fluid neighbours occupy slots [0, nf); wall neighbours start at the next
// quad boundary, wall_slot0(nf) = 4 ceil(nf / 4).
namespace sph {
__device__ __forceinline__ int64_t slot_index(int64_t n, int64_t i, int s) {
  return ((int64_t)(s >> 2) * n + i) * 4 + (s & 3);
}
__device__ __forceinline__ int wall_slot0(int nf) { return (nf + 3) & ~3; }
}  // namespace sph
