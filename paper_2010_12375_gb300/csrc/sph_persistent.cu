// Persistent substep loop: one cooperative launch runs every acoustic substep of an
// advection step for every tank of a handle (the batched form of many uneven tanks in one
// launch over the flattened particle index), instead of three launches per substep.
//
// Per substep, in three phases separated by grid-wide barriers:
//   dt         block 0 runs Eq. dt-relax for every tank (the block body the per-launch
//              k_dt_acoustic runs) and records whether any tank needs another substep
//   pressure   every block walks its grid-stride share of the particles through the
//              pressure relaxation (the same per-particle code as k_pressure_relaxation)
//   density    likewise the density relaxation
// and the loop ends after the substep in which the last tank covered its Dt_ad. Results are
// bit-identical to the per-launch loop: the same per-particle arithmetic, and |v|max is a
// maximum (order-free).
//
// Memory ordering: a phase gathers what other blocks wrote in the previous one, so the
// state arrays are read through plain (coherent) loads, never the read-only path, and the
// barrier fences before arriving and after leaving. The barrier's wait is bounded: a block
// that waits longer than about a second sets ERR_TIMEOUT and returns, and the others then
// time out at their next barrier, so the launch always ends. The launch is cooperative,
// which makes the runtime refuse a grid larger than can be resident at once.
#include <algorithm>

#include "sph_ctrl.cuh"
#include "sph_grid_sync.cuh"
#include "sph_relax.cuh"

namespace sph {
namespace {

constexpr int kPBlock = 128;

// |v^{n+1}|^2 maximum per tank: one atomic per warp when its particles share a tank.
__device__ __forceinline__ void warp_vmax(float v2, bool writer, int k, Ctrl* ctrl) {
  const unsigned full = 0xffffffffu;
  const int k0 = __shfl_sync(full, k, 0);
  if (__all_sync(full, k == k0)) {
    float m = writer ? v2 : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(full, m, o));
    const bool any = __any_sync(full, writer);
    if (any && (threadIdx.x & 31) == 0) atomicMax(&ctrl[k0].vmax2, __float_as_uint(m));
  } else if (writer) {
    atomicMax(&ctrl[k].vmax2, __float_as_uint(v2));
  }
}

template <int D, bool PER, bool UNI, bool TV>
__global__ void __launch_bounds__(kPBlock, 6)
k_substeps_persistent(const Inst Ip, int64_t n, int n_inst, const Inst* __restrict__ inst, Ctrl* ctrl, Global* g,
                      GridBarrier* bar, int4* PS, float4* VS, int4* PH, float4* VH, const float* __restrict__ mass,
                      const int* __restrict__ inst_of, const int* __restrict__ nbr,
                      const uint32_t* __restrict__ nbc, const int4* __restrict__ WP,
                      const float4* __restrict__ WN, const float4* __restrict__ acc_prior,
                      float4* __restrict__ acc_keep) {
  const int64_t stride = (int64_t)gridDim.x * kPBlock;
  for (int it = 0;; ++it) {
    if (blockIdx.x == 0) {
      const int any = dt_acoustic_block(n_inst, inst, ctrl, g);
      if (threadIdx.x == 0) {
        bar->active[it & 1] = any;           // the slot the others read after this substep
        g->active = any;
        g->substeps += 1;
      }
    }
    if (!grid_barrier(bar, g)) return;
    for (int64_t i0 = (int64_t)blockIdx.x * kPBlock; i0 < n; i0 += stride) {
      const int64_t i = i0 + threadIdx.x;
      bool valid = i < n;
      const int k = inst_index(inst_of, valid ? i : n - 1);
      const double dtd = __ldcg(&ctrl[k].dt);
      if (dtd == 0.0) valid = false;
      const Inst& I = UNI ? Ip : inst[k];
      bool writer;
      const float v2 = pr_particle<D, PER, 1, false, TV, const int4*, const float4*>(
          I, i, 0, valid, dtd, nullptr, n, PS, VS, PH, VH, mass, nbr, nbc, WP, WN, acc_prior, acc_keep, g, &writer);
      warp_vmax(v2, writer, k, ctrl);
    }
    if (!grid_barrier(bar, g)) return;
    for (int64_t i0 = (int64_t)blockIdx.x * kPBlock; i0 < n; i0 += stride) {
      const int64_t i = i0 + threadIdx.x;
      bool valid = i < n;
      const int k = inst_index(inst_of, valid ? i : n - 1);
      const double dtd = __ldcg(&ctrl[k].dt);
      if (dtd == 0.0) valid = false;
      if (!valid) continue;
      const Inst& I = UNI ? Ip : inst[k];
      dr_particle<D, PER, 1, false, const int4*, const float4*>(I, i, 0, true, dtd, nullptr, n, PH, VH, PS, VS,
                                                               mass, nbr, nbc, WP, WN, g);
    }
    if (!grid_barrier(bar, g)) return;
    if (!__ldcg(&bar->active[it & 1])) break;
  }
}

template <int D, bool PER, bool UNI, bool TV>
cudaError_t launch_persistent_t(const Buffers& b, cudaStream_t s, int* grid_out) {
  auto kern = k_substeps_persistent<D, PER, UNI, TV>;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess && !coop) e = cudaErrorNotSupported;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPBlock, 0);
  if (e != cudaSuccess) return e;
  const int64_t want = (b.n + kPBlock - 1) / kPBlock;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * sms));
  *grid_out = grid;
  Inst Ip = b.inst0;
  int64_t n = b.n;
  int n_inst = b.n_inst;
  const Inst* inst = b.inst;
  Ctrl* ctrl = b.ctrl;
  Global* g = b.glob;
  GridBarrier* bar = b.pbar;
  int4* PS = b.PS;
  float4* VS = b.VS;
  int4* PH = b.PH;
  float4* VH = b.VH;
  const float* mass = b.mass;
  const int* inst_of = b.inst_of;
  const int* nbr = b.nbr;
  const uint32_t* nbc = b.nbc;
  const int4* WP = b.nw ? b.WP : nullptr;
  const float4* WN = b.nw ? b.WN : nullptr;
  const float4* acc_prior = b.acc_prior;
  float4* acc_keep = b.acc_keep;
  void* args[] = {&Ip, &n, &n_inst, &inst, &ctrl, &g, &bar, &PS, &VS, &PH, &VH, &mass, &inst_of, &nbr, &nbc,
                  &WP, &WN, &acc_prior, &acc_keep};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kPBlock), args, 0, s);
}

template <int D, bool PER>
cudaError_t launch_persistent_d(const Buffers& b, cudaStream_t s, int* grid_out) {
  const bool uni = b.n_inst == 1;
  if (b.any_transport)
    return uni ? launch_persistent_t<D, PER, true, true>(b, s, grid_out)
               : launch_persistent_t<D, PER, false, true>(b, s, grid_out);
  return uni ? launch_persistent_t<D, PER, true, false>(b, s, grid_out)
             : launch_persistent_t<D, PER, false, false>(b, s, grid_out);
}

}  // namespace

cudaError_t launch_substeps_persistent(const Buffers& b, cudaStream_t s, int* grid_out) {
  *grid_out = 0;
  cudaError_t e = cudaMemsetAsync(&b.pbar->count, 0, sizeof(unsigned), s);   // a clean start after a timeout
  if (e != cudaSuccess) return e;
  if (b.dim == 2) return b.any_periodic ? launch_persistent_d<2, true>(b, s, grid_out)
                                        : launch_persistent_d<2, false>(b, s, grid_out);
  return b.any_periodic ? launch_persistent_d<3, true>(b, s, grid_out) : launch_persistent_d<3, false>(b, s, grid_out);
}

}  // namespace sph
