// Acoustic time-step control of one substep (Eq. dt-relax), shared by the per-launch
// kernel (k_dt_acoustic) and the persistent substep loop.
#pragma once
#include "sph_common.cuh"

namespace sph {

// Run by all threads of one block: for every tank not yet done, dt = min(cfl_ac h /
// (c0 + |v|max), Dt_ad - tau), advance tau and t, and mark the tank done once its Dt_ad is
// covered; a done tank gets dt = 0 (its particles sit this substep out). A non-finite or
// vanishing step sets ERR_DT, a substep count beyond the tank's bound ERR_TIMEOUT, and
// either ends the tank's loop instead of letting a device-side loop spin. Returns, in every
// thread, whether some tank still needs substeps after this one.
// dt_cap (or NULL): per tank, a cap on the acoustic step (0 = none), written by a coupled
// solid run with single time stepping.
__device__ __forceinline__ int dt_acoustic_block(int n_inst, const Inst* __restrict__ inst, Ctrl* ctrl, Global* g,
                                                 const double* dt_cap = nullptr) {
  int any = 0;
  for (int k = threadIdx.x; k < n_inst; k += blockDim.x) {
    const Inst& I = inst[k];
    Ctrl& C = ctrl[k];
    if (C.done) {
      C.dt = 0.0;
      continue;
    }
    double vmax = sqrt((double)__uint_as_float(C.vmax2));
    C.vmax2 = 0u;                                   // refilled by the pressure relaxation
    double dt_ac = I.cfl_ac * I.h_d / (I.c0_d + vmax);
    if (dt_cap && dt_cap[k] > 0.0) dt_ac = fmin(dt_ac, dt_cap[k]);
    double rem = C.dt_ad - C.tau;
    double dt = fmin(dt_ac, rem);
    if (!(dt_ac > 1e-12 * I.h_d / I.c0_d) || !(rem > 0.0) || !(dt > 0.0)) {
      atomicOr(&g->err, ERR_DT);
      C.dt = 0.0;
      C.done = 1;
      continue;
    }
    if (C.sub_in_step >= I.max_sub) {
      atomicOr(&g->err, ERR_TIMEOUT);
      C.dt = 0.0;
      C.done = 1;
      continue;
    }
    C.dt = dt;
    C.tau += dt;
    C.t += dt;
    C.substeps += 1;
    C.sub_in_step += 1;
    if (C.tau >= C.dt_ad * (1.0 - kLoopSlack)) C.done = 1;
    else any = 1;
  }
  return __syncthreads_or(any);
}

}  // namespace sph
