// FP64 diagnostics for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's
// device memory pool or under a fixed device-memory budget, and hosts that forbid
// any runtime allocation once they have started. sph_diagnostics needs a handle,
// and creating a handle allocates. sph_diagnostics_noalloc computes the same
// conservation diagnostics from the caller's own device arrays. Its only scratch
// is a fixed array in the library's device image (a file-scope __device__
// variable), so the call itself allocates nothing.
//
// The scratch holds one row of partial sums per block plus the final row. The
// grid never exceeds kNaBlocks blocks (a grid-stride loop covers any n), so the
// scratch size is fixed: (1024 + 1) x 16 doubles = 131,200 bytes, held by every
// GPU that loads the library until the process exits. Every call overwrites all
// the rows it reads, so nothing has to be cleared between calls; calls that
// overlap on the GPU (two streams, or two threads) share the array and race.
// The first call on each device looks up the array's device address with that
// device current; make that first call before any stream capture begins.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "sph.h"

namespace {

constexpr int kNaBlocks = 1024;
constexpr int kNaThreads = 256;
constexpr int kNaFields = 16;
constexpr int kNaMaxDevices = 64;
constexpr int64_t kNaMaxParticles = 2147483647;   // 2^31 - 1

static __device__ __align__(256) double g_noalloc_scratch[kNaBlocks * kNaFields + kNaFields];

std::mutex g_setup_mutex;
double* g_scratch_addr[kNaMaxDevices] = {nullptr};

enum { F_MASS = 0, F_PX, F_PY, F_PZ, F_KE, F_PE, F_IE, F_SUMDEV, F_MAXDEV, F_MAXX, F_COUNT };
constexpr int kSums = 8;

thread_local std::string t_last_error;

int fail(int code, const char* msg) {
  t_last_error = msg;
  return code;
}

// Per-block partials of the diagnostics over a grid-stride range of particles.
__global__ void __launch_bounds__(kNaThreads)
k_noalloc_partial(int64_t n, int dim, const double* __restrict__ pos, const double* __restrict__ vel,
                  const double* __restrict__ rho, const double* __restrict__ mass, double g0, double g1,
                  double g2, double rho0, double c0, double* __restrict__ scratch) {
  double acc[kSums];
#pragma unroll
  for (int f = 0; f < kSums; ++f) acc[f] = 0.0;
  double maxdev = 0.0, maxx = -1e300, cnt = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double m = mass[i];
    const double vx = vel[i * dim], vy = vel[i * dim + 1], vz = dim == 3 ? vel[i * dim + 2] : 0.0;
    const double x = pos[i * dim], y = pos[i * dim + 1], z = dim == 3 ? pos[i * dim + 2] : 0.0;
    const double dev = rho[i] / rho0 - 1.0;
    acc[F_MASS] += m;
    acc[F_PX] += m * vx;
    acc[F_PY] += m * vy;
    acc[F_PZ] += m * vz;
    acc[F_KE] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    acc[F_PE] -= m * (g0 * x + g1 * y + g2 * z);
    acc[F_IE] += m * c0 * c0 * (log1p(dev) - dev / (1.0 + dev));
    acc[F_SUMDEV] += fabs(dev);
    maxdev = fmax(maxdev, fabs(dev));
    maxx = fmax(maxx, x);
    cnt += 1.0;
  }
  __shared__ double red[kNaThreads];
  double* out = scratch + (size_t)blockIdx.x * kNaFields;
  for (int f = 0; f < kNaFields; ++f) {
    double v = f < kSums ? acc[f] : (f == F_MAXDEV ? maxdev : (f == F_MAXX ? maxx : (f == F_COUNT ? cnt : 0.0)));
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = kNaThreads / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double o = red[threadIdx.x + s];
        red[threadIdx.x] = (f == F_MAXDEV || f == F_MAXX) ? fmax(red[threadIdx.x], o) : red[threadIdx.x] + o;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = red[0];
    __syncthreads();
  }
}

// Ordered sum of the partials of this call's blocks into the final row.
__global__ void k_noalloc_final(int blocks, double* __restrict__ scratch) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double r[kNaFields];
  for (int f = 0; f < kNaFields; ++f) r[f] = f == F_MAXX ? -1e300 : 0.0;
  for (int b = 0; b < blocks; ++b)
    for (int f = 0; f < kNaFields; ++f) {
      double v = scratch[(size_t)b * kNaFields + f];
      r[f] = (f == F_MAXDEV || f == F_MAXX) ? fmax(r[f], v) : r[f] + v;
    }
  for (int f = 0; f < kNaFields; ++f) scratch[(size_t)kNaBlocks * kNaFields + f] = r[f];
}

// Device memory of the current device, or managed memory: the kernels run on the current
// device and read the arrays directly. Device memory of another GPU is refused (its
// addresses are not this device's, and the scratch address is looked up per device).
bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  int cur = -1;
  if (at.type != cudaMemoryTypeDevice || cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.device == cur;
}

// Device address of the scratch array on the current device, looked up once per
// device with that device current.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPH_E_CUDA, "sph_diagnostics_noalloc: no current CUDA device");
  }
  if (dev < 0 || dev >= kNaMaxDevices) return fail(SPH_E_INVALID, "sph_diagnostics_noalloc: device index too large");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(SPH_E_CUDA, "sph_diagnostics_noalloc: cudaGetSymbolAddress of the static scratch failed");
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return SPH_OK;
}

}  // namespace

const char* sph_noalloc_last_error() { return t_last_error.c_str(); }

extern "C" int sph_diagnostics_noalloc(const sph_params* p, int64_t n, const double* pos,
                                       const double* vel, const double* rho, const double* mass,
                                       sph_diag* out, void* stream) {
  if (!p || !out) return fail(SPH_E_INVALID, "sph_diagnostics_noalloc: params and out are required");
  if (p->dim != 2 && p->dim != 3) return fail(SPH_E_INVALID, "sph_diagnostics_noalloc: dim must be 2 or 3");
  if (!(p->rho0 > 0.0) || !std::isfinite(p->c0)) return fail(SPH_E_INVALID, "sph_diagnostics_noalloc: bad rho0 or c0");
  if (n < 0 || n > kNaMaxParticles)
    return fail(SPH_E_INVALID, "sph_diagnostics_noalloc: n must be in [0, 2^31 - 1]");
  if (n > 0 && (!pos || !vel || !rho || !mass))
    return fail(SPH_E_INVALID, "sph_diagnostics_noalloc: pos, vel, rho and mass are required");
  if (n > 0 && (!on_device(pos) || !on_device(vel) || !on_device(rho) || !on_device(mass)))
    return fail(SPH_E_INVALID, "sph_diagnostics_noalloc: arrays must be device memory of the current device");
  double* scratch = nullptr;
  int r = scratch_address(&scratch);
  if (r != SPH_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t want = (n + kNaThreads * 8 - 1) / (kNaThreads * 8);
  int blocks = (int)(want < 1 ? 1 : (want > kNaBlocks ? kNaBlocks : want));
  k_noalloc_partial<<<blocks, kNaThreads, 0, s>>>(n, p->dim, pos, vel, rho, mass, p->gravity[0],
                                                  p->gravity[1], p->dim == 3 ? p->gravity[2] : 0.0,
                                                  p->rho0, p->c0, scratch);
  cudaError_t le = cudaGetLastError();
  if (le == cudaSuccess) {
    k_noalloc_final<<<1, 1, 0, s>>>(blocks, scratch);
    le = cudaGetLastError();
  }
  if (le != cudaSuccess)      // the result row would be a previous call's: report, do not read
    return fail(SPH_E_CUDA, "sph_diagnostics_noalloc: kernel launch failed");
  double v[kNaFields];
  cudaError_t e = cudaMemcpyAsync(v, scratch + (size_t)kNaBlocks * kNaFields, sizeof(v),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SPH_E_CUDA, "sph_diagnostics_noalloc: kernel or copy failed");
  }
  sph_diag d;
  d.mass = v[F_MASS];
  d.momentum[0] = v[F_PX];
  d.momentum[1] = v[F_PY];
  d.momentum[2] = v[F_PZ];
  d.kinetic = v[F_KE];
  d.potential = v[F_PE];
  d.internal = v[F_IE];
  d.energy = v[F_KE] + v[F_PE] + v[F_IE];
  d.n_fluid = (int64_t)v[F_COUNT];
  d.max_rho_dev = v[F_MAXDEV];
  d.mean_rho_dev = d.n_fluid ? v[F_SUMDEV] / (double)d.n_fluid : 0.0;
  d.front_x = d.n_fluid ? v[F_MAXX] : 0.0;
  d.t = 0.0;
  d.dt_ad = 0.0;
  d.advection_steps = 0;
  d.substeps = 0;
  *out = d;
  return SPH_OK;
}
