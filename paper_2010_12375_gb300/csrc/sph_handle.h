// Library-side definition of the opaque sph_handle (shared by the C-ABI translation units).
#pragma once
#include <string>
#include <vector>

#include "sph.h"
#include "sph_kernels.h"

struct sph_handle {
  sph::Buffers b;
  std::vector<sph_params> params;
  std::vector<sph::Inst> hinst;
  uint32_t flags = 0;
  std::string err;
  std::vector<void*> allocs;
  int64_t device_bytes = 0;
  int64_t launches = 0;            // kernels launched directly by the host
  int64_t graph_kernels = 0;       // kernels executed by graph launches
  // graph of one advection step
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int64_t graph_fixed = 0, graph_body = 0;
  cudaStream_t cap_stream = nullptr;
  // staging and host mirrors
  double* stage = nullptr;
  size_t stage_elems = 0;
  double* diag_scratch = nullptr;
  double* diag_out = nullptr;
  sph::Global* hglob = nullptr;         // pinned host mirror of the device status
  // kernel timing
  bool timing = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  // chunked host upload of sph_set_state: copies on their own stream, the import of
  // each chunk on the caller's stream as soon as the chunk has arrived
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_ev[9] = {nullptr};
  double ms[2] = {0.0, 0.0};
  int64_t timed[2] = {0, 0};
  bool cells_valid = false;
  bool rows_valid = false;         // row pieces match the current cell order (row-task form)
  float4* grad = nullptr;          // [3][n] gradient sums of sph_gradient_diagnostics (lazily)
  sph_solid* solid = nullptr;      // attached elastic solid (sph_solid_create), or NULL
};

// Host-side helpers of sph_api.cu used by the other C-ABI translation units.
int sph_sync_status(sph_handle* h, cudaStream_t s);
// SPH_FLAG_DEBUG_BOUNDS: check the cell offsets and the neighbour table before a kernel reads
// them (synchronous); SPH_OK at once when the flag is off.
int sph_debug_check(sph_handle* h, cudaStream_t s);
// Drop the captured graph of an advection step (the loop's kernels changed).
void sph_drop_graph(sph_handle* h);
// Fluid-structure coupling hooks of the fluid's loop (sph_fsi.cu), no-ops without a solid:
// the near-fluid list after a configuration update, the coupling forces after the pressure
// relaxation, the continuity term and the solid's steps after the density relaxation.
void sph_fsi_after_build(sph_handle* h, cudaStream_t s, int64_t* launches);
void sph_fsi_after_pressure(sph_handle* h, cudaStream_t s, int64_t* launches);
void sph_fsi_after_density(sph_handle* h, cudaStream_t s, int64_t* launches);
void sph_fsi_set_gravity(sph_handle* h, const double* g);   // the attached solid's gravity, if any
