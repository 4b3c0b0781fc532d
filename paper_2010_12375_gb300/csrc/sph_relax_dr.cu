// Density relaxation launches (kernels and pair terms in sph_relax.cuh). Its own
// translation unit so the two relaxation kernels compile in parallel.
#include "sph_relax.cuh"

namespace sph {

void launch_density_relaxation(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  const int tpp = b.cfg.dr_tpp;
  int block = b.cfg.dr_block;
  if (row_form(block)) {
    if (!b.row_task || b.geo) {
      block = 128;                        // row pieces exist for one tank only
    } else if (!*b.rows_valid) {           // first row-task launch since the cells changed
      launch_row_tasks(b, s, launches);
      *b.rows_valid = true;
    }
  }
  if (b.dim == 2) {
    if (b.any_periodic) launch_dr<2, true>(tpp, block, b, s);
    else launch_dr<2, false>(tpp, block, b, s);
  } else {
    if (b.any_periodic) launch_dr<3, true>(tpp, block, b, s);
    else launch_dr<3, false>(tpp, block, b, s);
  }
  ++*launches;
}

}  // namespace sph
