// FP64 conservation diagnostics of each tank: mass, momentum, kinetic energy,
// potential energy -sum m g.r, internal energy of the EoS p = c0^2 (rho - rho0)
// (per unit mass c0^2 (ln(rho/rho0) + rho0/rho - 1)), density deviation and
// front position. Two passes with a fixed summation order, so the result is
// bit-reproducible: per-block partials, then one ordered sum per instance.
#include "sph_kernels.h"

namespace sph {

namespace {

constexpr int kDiagBlock = 256;
constexpr int kMaxBlocksPerInst = 512;

enum { F_MASS = 0, F_PX, F_PY, F_PZ, F_KE, F_PE, F_IE, F_SUMDEV, F_MAXDEV, F_MAXX, F_COUNT };
constexpr int kSumFields = 8;   // fields 0..7 are sums, 8..9 maxima, 10 count

int blocks_per_inst(const Buffers& b) {
  int64_t per = b.n_inst ? (b.n + b.n_inst - 1) / b.n_inst : 0;
  int64_t want = (per + kDiagBlock * 2 - 1) / (kDiagBlock * 2);
  if (b.n_inst == 1) want = (b.n + kDiagBlock * 2 - 1) / (kDiagBlock * 2);
  if (want < 1) want = 1;
  if (want > kMaxBlocksPerInst) want = kMaxBlocksPerInst;
  return (int)want;
}

// ln(1 + e) - e / (1 + e), the EoS energy per unit mass over c0^2 at rho/rho0 = 1 + e:
// for |e| <= 1/20 its Taylor series sum_{k>=2} (-1)^k (k-1)/k e^k to k = 16 (the remainder
// is below 1e-18 of the sum), else the closed form.
__device__ __forceinline__ double eos_energy(double e) {
  if (fabs(e) > 0.05) return log1p(e) - e / (1.0 + e);
  double s = -15.0 / 16.0;                            // coefficient of e^16
#pragma unroll
  for (int k = 15; k >= 2; --k) s = fma(s, e, (k & 1 ? -1.0 : 1.0) * (double)(k - 1) / (double)k);
  return s * e * e;
}

template <int D>
__global__ void __launch_bounds__(kDiagBlock)
k_diag_partial(const int4* __restrict__ P, const float4* __restrict__ V, const float* __restrict__ mass,
               const Inst* __restrict__ inst, double* __restrict__ part) {
  const int k = blockIdx.y;
  const Inst& I = inst[k];
  double acc[kSumFields];
#pragma unroll
  for (int f = 0; f < kSumFields; ++f) acc[f] = 0.0;
  double maxdev = 0.0, maxx = -1e300, cnt = 0.0;
  for (long long i = I.fluid_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < I.fluid_end;
       i += (long long)gridDim.x * blockDim.x) {
    const int4 p = P[i];
    const float4 v = V[i];
    const double m = mass ? (double)mass[i] : (double)I.mass;
    const double vx = v.x, vy = v.y, vz = D == 3 ? (double)v.z : 0.0;
    const double x = I.lo[0] + (double)p.x * I.dq_d;
    const double y = I.lo[1] + (double)p.y * I.dq_d;
    const double z = D == 3 ? I.lo[2] + (double)p.z * I.dq_d : 0.0;
    const double dev = (double)i2f(p.w) / I.rho0_d;            // rho/rho0 - 1
    acc[F_MASS] += m;
    acc[F_PX] += m * vx;
    acc[F_PY] += m * vy;
    acc[F_PZ] += m * vz;
    acc[F_KE] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    acc[F_PE] -= m * ((double)I.g[0] * x + (double)I.g[1] * y + (double)I.g[2] * z);
    acc[F_IE] += m * I.c0_d * I.c0_d * eos_energy(dev);
    acc[F_SUMDEV] += fabs(dev);
    maxdev = fmax(maxdev, fabs(dev));
    maxx = fmax(maxx, x);
    cnt += 1.0;
  }
  // block total per field: a fixed butterfly in each warp, then the warp totals in order
  __shared__ double red[kDiagFields][kDiagBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int f = 0; f < kDiagFields; ++f) {
    const bool is_max = (f == F_MAXDEV || f == F_MAXX);
    double val = f < kSumFields ? acc[f] : (f == F_MAXDEV ? maxdev : (f == F_MAXX ? maxx : (f == F_COUNT ? cnt : 0.0)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, val, o);
      val = is_max ? fmax(val, other) : val + other;
    }
    if (lane == 0) red[f][warp] = val;
  }
  __syncthreads();
  if (threadIdx.x < kDiagFields) {
    const int f = threadIdx.x;
    const bool is_max = (f == F_MAXDEV || f == F_MAXX);
    double r = red[f][0];
    for (int w = 1; w < kDiagBlock / 32; ++w) r = is_max ? fmax(r, red[f][w]) : r + red[f][w];
    part[((size_t)k * gridDim.x + blockIdx.x) * kDiagFields + f] = r;
  }
}

// Per instance: one 256-thread block; thread t sums field t % 16 over the blocks
// t / 16, t / 16 + 16, ... in order, then the 16 group sums of each field are added in
// order: a fixed summation order, independent of scheduling.
__global__ void __launch_bounds__(256)
k_diag_final(int n_inst, int bpi, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double grp[16][kDiagFields];
  const int k = blockIdx.x;
  const int f = threadIdx.x % kDiagFields, g = threadIdx.x / kDiagFields;
  const bool is_max = (f == F_MAXDEV || f == F_MAXX);
  double r = f == F_MAXX ? -1e300 : 0.0;
  for (int b = g; b < bpi; b += 16) {
    const double v = part[((size_t)k * bpi + b) * kDiagFields + f];
    r = is_max ? fmax(r, v) : r + v;
  }
  grp[g][f] = r;
  __syncthreads();
  if (threadIdx.x < kDiagFields) {
    double t = grp[0][f];
    for (int q = 1; q < 16; ++q) t = is_max ? fmax(t, grp[q][f]) : t + grp[q][f];
    out[(size_t)k * kDiagFields + f] = t;
  }
}

}  // namespace

size_t diag_scratch_elems(const Buffers& b) {
  return (size_t)b.n_inst * kMaxBlocksPerInst * kDiagFields;
}

void launch_diagnostics(const Buffers& b, double* scratch, double* out, cudaStream_t s,
                        int64_t* launches) {
  int bpi = blocks_per_inst(b);
  dim3 grid(bpi, b.n_inst);
  if (b.dim == 2)
    k_diag_partial<2><<<grid, kDiagBlock, 0, s>>>(b.PS, b.VS, b.mass, b.inst, scratch);
  else
    k_diag_partial<3><<<grid, kDiagBlock, 0, s>>>(b.PS, b.VS, b.mass, b.inst, scratch);
  k_diag_final<<<b.n_inst, 256, 0, s>>>(b.n_inst, bpi, scratch, out);
  *launches += 2;
}

}  // namespace sph
