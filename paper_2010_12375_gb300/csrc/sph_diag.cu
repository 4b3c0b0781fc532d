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
  int64_t want = (per + kDiagBlock * 8 - 1) / (kDiagBlock * 8);
  if (b.n_inst == 1) want = (b.n + kDiagBlock * 8 - 1) / (kDiagBlock * 8);
  if (want < 1) want = 1;
  if (want > kMaxBlocksPerInst) want = kMaxBlocksPerInst;
  return (int)want;
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
    acc[F_IE] += m * I.c0_d * I.c0_d * (log1p(dev) - dev / (1.0 + dev));
    acc[F_SUMDEV] += fabs(dev);
    maxdev = fmax(maxdev, fabs(dev));
    maxx = fmax(maxx, x);
    cnt += 1.0;
  }
  __shared__ double red[kDiagBlock];
  double* out = part + ((size_t)k * gridDim.x + blockIdx.x) * kDiagFields;
  for (int f = 0; f < kDiagFields; ++f) {
    double val = f < kSumFields ? acc[f] : (f == F_MAXDEV ? maxdev : (f == F_MAXX ? maxx : (f == F_COUNT ? cnt : 0.0)));
    red[threadIdx.x] = val;
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double o = red[threadIdx.x + s];
        if (f == F_MAXDEV || f == F_MAXX) red[threadIdx.x] = fmax(red[threadIdx.x], o);
        else red[threadIdx.x] += o;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = red[0];
    __syncthreads();
  }
}

__global__ void k_diag_final(int n_inst, int bpi, const double* __restrict__ part, double* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_inst; k += gridDim.x * blockDim.x) {
    double r[kDiagFields];
    for (int f = 0; f < kDiagFields; ++f) r[f] = (f == F_MAXX) ? -1e300 : 0.0;
    for (int b = 0; b < bpi; ++b) {
      const double* p = part + ((size_t)k * bpi + b) * kDiagFields;
      for (int f = 0; f < kDiagFields; ++f) {
        if (f == F_MAXDEV || f == F_MAXX) r[f] = fmax(r[f], p[f]);
        else r[f] += p[f];
      }
    }
    for (int f = 0; f < kDiagFields; ++f) out[(size_t)k * kDiagFields + f] = r[f];
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
  k_diag_final<<<(b.n_inst + 127) / 128, 128, 0, s>>>(b.n_inst, bpi, scratch, out);
  *launches += 2;
}

}  // namespace sph
