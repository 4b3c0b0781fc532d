// Host-side launch interface of the WCSPH kernels (internal to libsph.so).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_common.cuh"

namespace sph {

// Launch configuration of the acoustic-substep kernels (chosen by the autotuner):
// threads per particle (1, 2, 4) and block size (128, 256, 512), or the row-task form
// (one thread per particle, block kRowBlock): one resident block of kRowWarps warps an SM,
// each warp taking 32-particle pieces of one search-cell row from its block's queue.
constexpr int kRowWarps = 28;
constexpr int kRowBlock = kRowWarps * 32;
struct LaunchCfg {
  int pr_tpp = 1, pr_block = 256;   // pressure relaxation
  int dr_tpp = 1, dr_block = 256;   // density relaxation
};

// Grid-wide barrier and loop flags of the persistent substep loop (device memory).
struct GridBarrier {
  unsigned count;      // blocks arrived at the current barrier
  unsigned gen;        // barriers completed
  int active[2];       // per substep (alternating): some tank needs another substep
};

// Device buffers of one handle. Fluid arrays are indexed in cell-sorted order.
struct Buffers {
  LaunchCfg cfg;
  int64_t n = 0, nw = 0, n_cells = 0;
  int n_inst = 1, dim = 2, cap = 0;
  bool any_periodic = false;      // some tank has a periodic axis
  bool any_transport = false;     // some tank has the transport velocity on
  Inst* inst = nullptr;           // [n_inst]
  Inst inst0{};                   // host copy of instance 0 (kernel argument when n_inst == 1)
  Ctrl* ctrl = nullptr;           // [n_inst]
  Global* glob = nullptr;         // [1]
  const int* inst_of = nullptr;   // [n] instance of each fluid slot (NULL when n_inst == 1)
  const int* winst_of = nullptr;  // [nw]
  int4* PS = nullptr;  float4* VS = nullptr;   // state between substeps
  int4* PH = nullptr;  float4* VH = nullptr;   // half step / reorder scratch
  float* mass = nullptr;          // [n] non-uniform masses, NULL when uniform per instance
  float* mass_tmp = nullptr;
  int* id = nullptr;              // [n] caller id of each sorted slot
  float4* acc_prior = nullptr;    // [n] viscous acceleration (NULL when inviscid)
  float4* acc_keep = nullptr;     // [n] last dv/dt (NULL unless kept)
  // cell build
  uint32_t* cell = nullptr;       // [n]
  uint32_t* rank = nullptr;       // [n]
  uint32_t* count = nullptr;      // [n_cells]
  uint32_t* fstart = nullptr;     // [n_cells + 1]
  int* key = nullptr;             // [n]
  int* src = nullptr;             // [n]
  uint32_t* scan_tmp = nullptr;   // scan block sums
  // walls
  int4* WP = nullptr;  float4* WN = nullptr;
  int* wid = nullptr;             // [nw] caller row of each sorted wall slot
  uint32_t* wstart = nullptr;     // [n_cells + 1]
  uint8_t* wnear = nullptr;       // [n_cells] 1: a wall particle lies within two search cells
  // neighbours (column-major ELL: nbr[k * n + i])
  int* nbr = nullptr;
  uint32_t* nbc = nullptr;        // [n] fluid count | wall count << 16
  float4* geo = nullptr;          // [cap][n] frozen r_i - r_j and (dW/dr)/r per slot (or NULL)
  GridBarrier* pbar = nullptr;    // [1] persistent substep loop
  double* dt_cap = nullptr;       // [n_inst] cap on the acoustic step (0 = none), or NULL
  // half-pair evaluation (or NULL): per-slot shares [cap][n], per-particle partial sums [n],
  // reverse slots [cap][n] (slot of j in i's row for each slot of j's row holding i < j)
  float4* hshare = nullptr;
  float4* hpart = nullptr;
  uint8_t* hrev = nullptr;
  // row tasks of the row-task launch form (one tank only; NULL otherwise): the pieces
  // (first slot, count <= 32) of every search-cell row along x, row after row
  int2* row_task = nullptr;       // [row_task_cap]
  uint32_t* row_cnt = nullptr;    // [n_rows] pieces of each row
  uint32_t* row_off = nullptr;    // [n_rows + 1] exclusive scan; row_off[n_rows] = pieces
  uint32_t* row_tmp = nullptr;    // scan scratch
  int64_t n_rows = 0, row_task_cap = 0;
  bool* rows_valid = nullptr;     // host flag: the pieces match the current cell order
  int n_sm = 0;                   // SMs of the device (grid of the row-task form)
};

size_t scan_tmp_elems(int64_t n);
void scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s,
                    int64_t* launches);

// cell build
void launch_hash(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_fluid_offsets(const Buffers& b, cudaStream_t s, int64_t* launches);   // scan of the counts
void launch_sort_fluid(const Buffers& b, cudaStream_t s, int64_t* launches);      // scatter, rank, reorder
// SPH_FLAG_DEBUG_BOUNDS checks: the fluid and wall cell offsets, the neighbour table
void launch_check_offsets(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_check_table(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_neighbours(const Buffers& b, cudaStream_t s, int64_t* launches);
// the row pieces of the row-task form from the current fluid cell offsets (one tank)
void launch_row_tasks(const Buffers& b, cudaStream_t s, int64_t* launches);
// whether a configured block selects the row-task form
inline bool row_form(int block) { return block == kRowBlock; }
void sort_walls(Buffers& b, int4* WP_tmp, float4* WN_tmp, int* wid_tmp, cudaStream_t s);
void flag_near_wall_cells(const Buffers& b, uint8_t* tmp, cudaStream_t s);
void launch_iota(int* a, int64_t n, cudaStream_t s);     // a[i] = i

// import / export
// rows [i0, i1) of the caller's arrays (i1 < 0: to the end)
void launch_import(const Buffers& b, const double* pos, const double* vel, const double* rho,
                   const double* drho, cudaStream_t s, int64_t i0 = 0, int64_t i1 = -1);
void launch_import_walls(const Buffers& b, const double* pos, const double* nrm, const double* vol,
                         cudaStream_t s);
void launch_export(const Buffers& b, double* pos, double* vel, double* rho, double* drho,
                   cudaStream_t s);
void launch_export_acc(const Buffers& b, double* acc, cudaStream_t s);
void launch_export_neighbours(const Buffers& b, int32_t* fc, int32_t* wc, int32_t* fids,
                              int32_t* wids, int32_t stride, cudaStream_t s);

// physics
void launch_pair_count(const Buffers& b, unsigned long long* out2, cudaStream_t s);
void launch_vmax(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_dt_advection(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_density(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_viscous(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_dt_acoustic(const Buffers& b, cudaStream_t s, cudaGraphConditionalHandle cond,
                        bool use_cond, int64_t* launches);
void launch_pressure_relaxation(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_density_relaxation(const Buffers& b, cudaStream_t s, int64_t* launches);
// every acoustic substep of the current advection step for every tank in one cooperative
// launch (not with the frozen-geometry reading); *grid_out receives the blocks launched
cudaError_t launch_substeps_persistent(const Buffers& b, cudaStream_t s, int* grid_out);
// half-pair evaluation: the reverse-slot map of the current table (after each build), and
// one relaxation (pressure or density) as its two passes
void launch_reverse_slots(const Buffers& b, cudaStream_t s, int64_t* launches);
void launch_half_pair(const Buffers& b, bool pressure, cudaStream_t s, int64_t* launches);
// per-slot pair geometry at the current positions, for the frozen-geometry reading
void launch_pair_geometry(const Buffers& b, cudaStream_t s, int64_t* launches);
// gather-only walk of the neighbour table (diagnostic), in the pressure relaxation's launch
// form (gather_rows: the row-task form); sink: one device word
void launch_gather_ceiling(const Buffers& b, unsigned* sink, cudaStream_t s, int64_t* launches);
bool gather_rows(const Buffers& b);

// diagnostics: out[n_inst * kDiagFields] doubles on the device
constexpr int kDiagFields = 16;
size_t diag_scratch_elems(const Buffers& b);
void launch_diagnostics(const Buffers& b, double* scratch, double* out, cudaStream_t s,
                        int64_t* launches);

}  // namespace sph
