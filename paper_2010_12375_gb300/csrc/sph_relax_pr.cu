// Pressure relaxation launches (kernels and pair terms in sph_relax.cuh). Its own
// translation unit so the two relaxation kernels compile in parallel.
#include "sph_relax.cuh"

namespace sph {

void launch_pressure_relaxation(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  const int tpp = b.cfg.pr_tpp, block = b.cfg.pr_block;
  if (b.dim == 2) {
    if (b.any_periodic) launch_pr<2, true>(tpp, block, b, s);
    else launch_pr<2, false>(tpp, block, b, s);
  } else {
    if (b.any_periodic) launch_pr<3, true>(tpp, block, b, s);
    else launch_pr<3, false>(tpp, block, b, s);
  }
  ++*launches;
}

}  // namespace sph
