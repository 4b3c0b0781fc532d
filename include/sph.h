/*
 * sph.h -- C ABI of the GB300 weakly-compressible SPH hot path (libsph.so).
 *
 * The library advances fluid particles with the Riemann-solver WCSPH scheme of
 * SPHinXsys (Zhang et al., arXiv 2010.12375): a cell-linked-list neighbour
 * search once per advection step, density re-initialisation (Eq. eqrhosum /
 * Eq. eqrhosumnosurface), the dual-criteria time steps (Eq. dt-advection,
 * Eq. dt-relax) and, per acoustic substep, the pressure and density relaxations
 * of the position-based Verlet scheme (Eqs. verlet-first-half,
 * verlet-first-mediate, verlet-first-final with Eq. riemannsph, Eq. eqeos and
 * the one-sided wall problem of Eqs. eqriepartial, eqrienoslip, eqriepright),
 * with a Wendland C2 kernel, dummy-particle walls and gravity; optionally the
 * transport velocity of Eq. transport (sph_params.p_transport) for flows without
 * free surface. A species carried by the fluid particles diffuses by Eq. grad-laplace
 * with two-stage Runge-Kutta steps (sph_species_*, sph_diffusion_step) and reacts by the
 * split QSS scheme of the reaction-diffusion models (sph_reaction_step).
 *
 * Conventions shared by every entry point
 *  - Return value: SPH_OK (0) or a negative SPH_E_* code. No call aborts the
 *    process or traps the GPU. After SPH_E_DOMAIN..SPH_E_TIMEOUT the handle
 *    stays valid for inspection (sph_get_state, sph_last_error).
 *  - Array arguments are plain pointers to host or device memory (unified
 *    addressing decides which); the library copies what it needs and never
 *    keeps a caller pointer beyond the call. Device arrays must belong to the
 *    current device (another GPU's memory returns SPH_E_INVALID). Vectors are
 *    interleaved per particle: pos[k*dim + a].
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *    asynchronous on it, except those that return host values, which
 *    synchronise that stream before returning.
 *  - Particle order at the boundary is always the caller's order ("id" order:
 *    row k is particle k). Inside, particles are re-sorted by search cell every
 *    advection step.
 *  - The handle is not thread safe; calls on one handle must be serialised.
 *
 * Position representation (part of the contract, so results can be checked
 * bit for bit): positions are held as fixed-point integers per axis,
 * q = rint((x - lo) / dq), with dq = cell / 2^bits, cell = 2h (or, when axes
 * are periodic, period / floor(period / 2h), all periodic axes sharing one
 * period), bits = min(22, 31 - bitlength(max cells per axis)). Particles are
 * stored by search cell, q >> (bits - 1) per axis (the cell halved on every axis),
 * flattened with x fastest, then by id. Particles j != i
 * are neighbours when sum_a (q_i,a - q_j,a)^2 < R2 (minimum image on periodic
 * axes), R2 = ceil((2h/dq)^2) evaluated in double precision: the integer
 * form of |r_i - r_j| < 2h.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define SPH_OK          0
#define SPH_E_INVALID  -1   /* bad argument or parameter (h <= 0, dim not 2/3, CFL <= 0, ...) */
#define SPH_E_CUDA     -2   /* a CUDA runtime call failed (message in sph_last_error)        */
#define SPH_E_OOM      -3   /* device allocation failed                                     */
#define SPH_E_DOMAIN   -4   /* a particle left the cell grid [lo, hi) on a non-periodic axis */
#define SPH_E_UNSTABLE -5   /* NaN/Inf in the state, or a time step below 1e-12 h/c0          */
#define SPH_E_CAPACITY -6   /* a particle has more neighbours than the per-particle capacity */
#define SPH_E_TIMEOUT  -7   /* a bounded device-side wait expired, or an advection step
                               needed more acoustic substeps than sph_params.max_substeps  */
#define SPH_E_BOUNDS   -8   /* SPH_FLAG_DEBUG_BOUNDS: a neighbour index, row count or cell
                               offset out of range, caught before any kernel used it      */

/* ---- flags (sph_params.flags) ----------------------------------------------------- */
#define SPH_FLAG_GRAPH     1u  /* sph_step runs each advection step as one CUDA graph whose
                                  acoustic-substep loop is a device-side conditional WHILE node */
#define SPH_FLAG_KEEP_ACC  2u  /* keep the last dv/dt of every particle for sph_get_acceleration */
#define SPH_FLAG_FROZEN_GEOMETRY 4u  /* keep each pair's vector r_i - r_j and (dW/dr)/r from the
                                      * configuration update (after sph_advection_step's density
                                      * re-initialisation) for every half step of the advection
                                      * step, as the neighbour relation of Sec. 6.2 stores them;
                                      * without it they are recomputed from the current
                                      * positions in every half step. Costs 16 B per neighbour
                                      * slot of device memory (n_fluid x capacity). */
#define SPH_FLAG_PERSISTENT  16u     /* sph_step runs all acoustic substeps of each advection step,
                                      * for every tank of the handle, in one cooperative
                                      * (persistent) launch: three phases per substep (time step,
                                      * pressure relaxation, density relaxation) separated by
                                      * grid-wide barriers whose waits are bounded (a timeout ends
                                      * the launch with SPH_E_TIMEOUT). Results are bit-identical
                                      * to the per-launch loop. Ignored with
                                      * SPH_FLAG_FROZEN_GEOMETRY, SPH_FLAG_HALF_PAIR,
                                      * SPH_FLAG_DEBUG_BOUNDS or kernel
                                      * timing on; takes precedence over SPH_FLAG_GRAPH. */
#define SPH_FLAG_HALF_PAIR   32u     /* evaluate every unordered fluid pair of the two relaxations
                                      * once (Newton's third law: P*_ij = P*_ji with the
                                      * antisymmetric kernel gradient of Eq. gradsph-weak; the
                                      * continuity term's velocity part symmetric, its pressure
                                      * part antisymmetric): a first pass adds each pair's share
                                      * for the lower particle and stores the upper particle's
                                      * share per neighbour slot, a second pass sums the stored
                                      * shares through a reverse-slot map built with each
                                      * configuration update. Fixed summation order, no atomics:
                                      * bit-reproducible; equal to the per-pair kernels up to
                                      * rounding. Costs 17 B per neighbour slot of device memory;
                                      * needs capacity <= 252; not with SPH_FLAG_FROZEN_GEOMETRY or
                                      * the transport velocity; the launch configuration and the
                                      * autotuner do not apply (one thread per particle). */
#define SPH_FLAG_DEBUG_BOUNDS 8u     /* check, before any kernel reads them, that the cell
                                      * offsets of every configuration update run from 0 to
                                      * the particle count without decreasing, and that every
                                      * neighbour row fits the capacity with every index in
                                      * range; a violation returns SPH_E_BOUNDS and launches
                                      * nothing that would read it. The checks synchronise
                                      * the stream, so sph_step then drives the loop from the
                                      * host (SPH_FLAG_GRAPH is ignored). */

typedef struct sph_handle sph_handle;   /* opaque, library-owned */

/* Problem parameters (one per tank). The paper's statement of the problem:
 * smoothing length h (Sec. 1.1), reference density rho0 and artificial sound
 * speed c0 of the EoS p = c0^2 (rho - rho0) (Eq. eqeos), advection and acoustic
 * CFL numbers (Sec. 2.4: 0.25 and 0.6), kinematic viscosity nu (Eq. eqviscous,
 * eta = rho0 nu; 0 = inviscid), gravity g (Eq. governingeq). */
typedef struct {
  int32_t  dim;           /* 2 or 3 */
  int32_t  free_surface;  /* 1: rho = max(rho*, rho0 sumW/sumW0) (Eq. eqrhosum); 0: without max */
  double   h;             /* smoothing length; kernel support radius is 2h                 */
  double   dp;            /* initial lattice spacing: sumW0 is the lattice sum at dp       */
  double   rho0, c0;      /* reference density, artificial sound speed                    */
  double   cfl_ad, cfl_ac;/* advection / acoustic CFL numbers                             */
  double   u_ref;         /* speed floor in Dt_ad = cfl_ad min(h / max(|v|max, u_ref), h^2/nu) */
  double   nu;            /* kinematic viscosity                                          */
  double   gravity[3];
  double   lo[3], hi[3];  /* cell-grid box (tank including its wall layers); unused axes ignored */
  int32_t  periodic[3];   /* 1 = periodic axis with period hi - lo (>= 3 cells)             */
  int32_t  capacity;      /* max neighbours (fluid + wall) per particle; 0 = 48 (2D) / 128 (3D) */
  uint32_t flags;         /* SPH_FLAG_* (taken from the first instance)                    */
  double   p_transport;   /* background pressure p0 of the transport velocity (Eq. transport,
                             flows without free surface); 0 = off. On: each pressure
                             relaxation also moves the mid-point position by dt^2/2 a_i,
                             a_i = -2 sum_j m_j p0 / (rho_i rho_j) grad_i W_ij over fluid
                             pairs at the mid-point; not with SPH_FLAG_FROZEN_GEOMETRY */
  int32_t  max_substeps;  /* bound of the device-side acoustic-substep loop of one advection
                             step (0 = 1000; a normal step takes 2-6): a step that needs more
                             stops there with SPH_E_TIMEOUT, the handle stays valid and
                             sph_clear_error lets it continue */
} sph_params;

/* FP64 conservation and bulk diagnostics of one tank. */
typedef struct {
  double  mass;           /* sum m                                                       */
  double  momentum[3];    /* sum m v                                                     */
  double  kinetic;        /* sum m |v|^2 / 2                                             */
  double  potential;      /* -sum m g . r                                                */
  double  internal;       /* sum m c0^2 (ln(rho/rho0) + rho0/rho - 1), the EoS energy     */
  double  energy;         /* kinetic + potential + internal                              */
  double  max_rho_dev;    /* max |rho/rho0 - 1|                                          */
  double  mean_rho_dev;   /* mean |rho/rho0 - 1|                                         */
  double  front_x;        /* max x over fluid particles                                  */
  double  t;              /* simulated time (FP64 accumulator)                           */
  double  dt_ad;          /* last advection step                                         */
  int64_t n_fluid;
  int64_t advection_steps;
  int64_t substeps;       /* acoustic substeps taken so far                              */
} sph_diag;

/* Sizes and derived constants of a handle. */
typedef struct {
  int32_t dim, n_instances, capacity, bits;
  int64_t n_fluid, n_wall, n_cells;  /* n_cells: search cells over all instances       */
  double  cell, dq, sigma0;        /* cell size, position quantum, lattice sumW0 (instance 0) */
  int64_t R2;                      /* integer neighbour threshold (instance 0)               */
  int64_t device_bytes;            /* device memory held by the handle                       */
} sph_info;

/* Check parameters on the host only (no GPU needed). SPH_OK or SPH_E_INVALID. */
int sph_params_check(const sph_params* p);

/* Create a handle holding n_instances independent tanks (1 = a single tank).
 * On failure *out may still receive a handle carrying the message for
 * sph_last_error; the caller destroys it.
 * Instance k owns fluid rows [fluid_offsets[k], fluid_offsets[k+1]) and wall rows
 * [wall_offsets[k], wall_offsets[k+1]); offsets may be NULL when n_instances = 1.
 * pos, vel: [n_fluid*dim] double; rho, mass: [n_fluid] double;
 * wall_pos, wall_normal: [n_wall*dim] double (unit normal pointing into the fluid);
 * wall_vol: [n_wall] double. All dims equal across instances. The walls are
 * static (wall velocity 0). d rho/dt starts at 0 and the simulated time at 0.
 * Walls are sorted into cells once here. *out receives the handle. */
int sph_create(const sph_params* params, int32_t n_instances,
               const int64_t* fluid_offsets, const int64_t* wall_offsets,
               int64_t n_fluid, const double* pos, const double* vel,
               const double* rho, const double* mass,
               int64_t n_wall, const double* wall_pos, const double* wall_normal,
               const double* wall_vol, void* stream, sph_handle** out);

void sph_destroy(sph_handle* h);

/* Message of the last failure on this handle ("" if none); with h = NULL, the
 * message of this thread's last failed sph_diagnostics_noalloc call. */
const char* sph_last_error(const sph_handle* h);

int sph_get_info(const sph_handle* h, sph_info* out);

/* Clear the handle's error state (the device error word and the message) after the caller
 * has inspected it, so that the next call does not report it again. Synchronous. */
int sph_clear_error(sph_handle* h, void* stream);

/* Overwrite one entry of the handle's internal tables (a test aid for SPH_FLAG_DEBUG_BOUNDS;
 * the paper has no counterpart). what = SPH_DEBUG_NEIGHBOUR: slot `slot` of the neighbour
 * row of the particle stored at position `index` in the library's current cell-sorted
 * order; what = SPH_DEBUG_WALL_OFFSET: entry `index` of the wall-particle cell offsets
 * (0..n_cells; kept from sph_create, read by every configuration update). Refused
 * (SPH_E_INVALID) unless the handle was created with SPH_FLAG_DEBUG_BOUNDS, since only then
 * is every table checked before a kernel reads it; an out-of-range index or slot is
 * SPH_E_INVALID too. Synchronous. */
#define SPH_DEBUG_NEIGHBOUR    1
#define SPH_DEBUG_WALL_OFFSET  2
int sph_debug_write(sph_handle* h, int32_t what, int64_t index, int32_t slot, int64_t value,
                    void* stream);

/* Configuration update (paper Sec. 2.4 / Sec. 6.2 mesh_cell_linked_list): hash
 * particles to search cells, sort by (search cell, id), cell offsets, reorder the state, and
 * build the neighbour set {j != i : |r_i - r_j| < 2h} of every fluid particle
 * (fluid and wall neighbours), frozen until the next call. */
int sph_build_cells(sph_handle* h, void* stream);

/* Start an advection step: Dt_ad (Eq. dt-advection, speed floor u_ref), density
 * re-initialisation (Eq. eqrhosum / Eq. eqrhosumnosurface; walls count in sum W,
 * sumW0 = lattice sum at dp including self) and the viscous acceleration
 * (Eq. eqviscous, fluid pairs, held over the substeps). Requires sph_build_cells
 * after the last position change. dt_ad_out (host, may be NULL) receives Dt_ad
 * of instance 0 and makes the call synchronous. */
int sph_advection_step(sph_handle* h, double* dt_ad_out, void* stream);

/* One acoustic substep for every instance whose advection step is not yet
 * covered: dt = min(cfl_ac h / (c0 + |v|max) (Eq. dt-relax), Dt_ad - tau), then
 * the pressure relaxation (Eq. verlet-first-half, Eq. eqeos, Eq. riemannsph
 * momentum with the wall problem, Eq. verlet-first-mediate) and the density
 * relaxation (Eq. verlet-first-final with Eq. riemannsph continuity).
 * Pair geometry is recomputed from the current positions; neighbours are the
 * frozen set. done_out (host, may be NULL) receives 1 once every instance has
 * covered its Dt_ad; dt_out (host, may be NULL) receives instance 0's dt. Either
 * makes the call synchronous. */
int sph_acoustic_substep(sph_handle* h, int32_t* done_out, double* dt_out, void* stream);

/* n_advection_steps complete dual-criteria steps: build cells, advection step,
 * substeps until Dt_ad is covered. With SPH_FLAG_GRAPH each step is one CUDA
 * graph launch (the substep loop is a device-side WHILE node); otherwise the
 * host drives the loop, synchronising once per substep. Synchronous. */
int sph_step(sph_handle* h, int32_t n_advection_steps, void* stream);

/* FP64 diagnostics, one sph_diag per instance into out[0..n_instances) (host). */
int sph_diagnostics(sph_handle* h, sph_diag* out, void* stream);

/* Copy the state out in id order: pos, vel [n_fluid*dim], rho, drho_dt [n_fluid]
 * (double; any pointer may be NULL). Positions are lo + q dq exactly. */
int sph_get_state(sph_handle* h, double* pos, double* vel, double* rho, double* drho_dt,
                  void* stream);

/* Replace the state (id order, same sizes as sph_create; drho_dt may be NULL = 0)
 * and, if t >= 0, instance 0's simulated time. Call sph_build_cells before
 * the next advection step (sph_step does). Host arrays of 262,144 particles or more are
 * copied in row chunks on a stream the handle owns, ordered after the work already on
 * `stream`, while `stream` converts each chunk that has arrived. Synchronous: the
 * caller's arrays may be reused when it returns. */
int sph_set_state(sph_handle* h, const double* pos, const double* vel, const double* rho,
                  const double* drho_dt, double t, void* stream);

/* Particle gradients of the density and the pressure of every fluid particle (Sec. 1.1,
 * "particle average and gradient"): the strong form of Eq. gradsph-strong, which gives the
 * local structure of a field, and the weak form of Eq. gradsph-weak, which conserves. The
 * paper's grad_i W_ij there is e_ij dW/dr with e_ij from i to j, minus the true gradient;
 * with the true grad_i W_ij = (dW/dr) (r_i - r_j)/|r_i - r_j| they read
 *   strong  grad f_i = sum_j V_j (f_j - f_i) grad_i W_ij,
 *   weak    grad f_i = sum_j V_j (f_i + f_j) grad_i W_ij,
 * over the neighbour set of the last configuration update (sph_build_cells or a step: call
 * sph_build_cells first for the set of the current positions) with the pair geometry of the
 * current positions; V_j = m_j/rho_j for fluid neighbours, and wall neighbours carry the
 * one-sided wall problem's p_w = p_i + rho_i g.(r_w - r_i), rho_w = rho0 + p_w/c0^2 and their
 * volume. Outputs: [n_fluid*dim] doubles each, caller order, host or device, any may be NULL.
 * FP32 sums with Kahan compensation. Synchronous. */
int sph_gradient_diagnostics(sph_handle* h, double* grad_rho_strong, double* grad_rho_weak,
                             double* grad_p_strong, double* grad_p_weak, void* stream);

/* dv/dt of the last pressure relaxation in id order [n_fluid*dim] (needs
 * SPH_FLAG_KEEP_ACC). */
int sph_get_acceleration(sph_handle* h, double* acc, void* stream);

/* Fluid ids in cell-sorted order after the last sph_build_cells [n_fluid]. */
int sph_get_permutation(sph_handle* h, int32_t* ids, void* stream);

/* Neighbour sets of the last sph_build_cells in id order: for fluid id i,
 * fluid_ids[i*stride .. +fluid_count[i]) holds fluid neighbour ids and
 * wall_ids[i*stride .. +wall_count[i]) wall row indices (caller order).
 * stride >= capacity. Order within a row is the library's traversal order. */
int sph_get_neighbours(sph_handle* h, int32_t* fluid_count, int32_t* wall_count,
                       int32_t* fluid_ids, int32_t* wall_ids, int32_t stride, void* stream);

/* Directed fluid-fluid and fluid-wall pairs in the neighbour sets of the last
 * sph_build_cells (host outputs; synchronous). */
int sph_pair_count(sph_handle* h, int64_t* fluid_pairs, int64_t* wall_pairs, void* stream);

/* Replace the gravity (the body force per unit mass, Eq. governingeq's g) of tank `instance`
 * (0-based; every tank when instance < 0) for every later call that advances the state, for
 * instance to follow a tank's translation in its own frame, g_eff(t) = g - a_tank(t). It
 * also enters the wall problem's P_R (Eq. eqriepright) and an attached solid's momentum
 * (the solid feels the same frame). A captured advection-step graph is rebuilt at its next
 * use. g: host array of 3 doubles (components beyond dim ignored). SPH_E_INVALID for a bad
 * instance or a non-finite component, the gravity unchanged. Synchronous. */
int sph_set_gravity(sph_handle* h, int32_t instance, const double* g, void* stream);

/* Launch configuration of the two acoustic-substep kernels: cfg[0] threads per particle
 * and cfg[1] block size of the pressure relaxation, cfg[2], cfg[3] the same for the
 * density relaxation. Threads per particle 1, 2 or 4 (the lanes of a particle split its
 * neighbour row and add their sums in a fixed order); block 128, 256 or 512; or, on a
 * handle of one tank, threads per particle 1 with block 896, the row-task form: one
 * resident block of 28 warps an SM, each warp taking the next 32 particles of one
 * search-cell row (the cells along x at fixed y, z) from its block's queue, the blocks
 * advancing through the cell order side by side; it computes each particle as the other
 * one-thread-per-particle variants do, so their results are identical bit for bit. Set
 * returns SPH_E_INVALID for other values. Handles created with SPH_FLAG_FROZEN_GEOMETRY
 * run one thread per particle in 128-thread blocks whatever the configuration says. */
int sph_get_launch_config(const sph_handle* h, int32_t* cfg);
int sph_set_launch_config(sph_handle* h, const int32_t* cfg);

/* Autotuner: runs one advection step, timing every launch variant of the two relaxation
 * kernels (3 x 3 threads-per-particle x block variants, and the row-task form on a handle
 * of one tank) on its first substep (each variant recomputes the same substep; the chosen
 * one writes the result), keeps the fastest, and records it in the cache file
 * $SPH_AUTOTUNE_CACHE (default $HOME/.cache/sph_gb300_autotune.json) under (GPU name, dim,
 * particle-count power of two, batched or single). sph_create applies a cached entry for
 * the same key. cfg_out (may be NULL) receives the chosen cfg; ms_out (may be NULL) 20
 * mean launch times, ms_out[10 kernel + 3 tpp_index + block_index] for the 3 x 3
 * variants and ms_out[10 kernel + 9] for the row-task form (-1 where it does not apply).
 * Synchronous. */
int sph_autotune(sph_handle* h, int32_t* cfg_out, double* ms_out, void* stream);

/* Gather ceiling (a measurement aid; the paper has no counterpart): times `reps` launches
 * of a kernel that walks the current neighbour table the way the pressure relaxation does
 * (one thread per particle in its configured launch form, per-particle blocks or row tasks,
 * 16-byte index quads, the 32-byte position + velocity record of every fluid neighbour and
 * the wall records gathered) with no pair arithmetic, and
 * writes the mean launch time in ms to *ms_out (host). No state is changed. Needs a
 * neighbour table (sph_build_cells or a step first: SPH_E_INVALID otherwise); reps >= 1.
 * Synchronous. */
int sph_gather_ceiling(sph_handle* h, int32_t reps, double* ms_out, void* stream);

/* Kernel launches the library has issued on this handle (graph nodes counted
 * once per execution, the substep loop by the device-side substep counter). */
int sph_kernel_launches(sph_handle* h, int64_t* out);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * each launch of the pressure and density relaxation kernels (host-driven loop
 * only; off by default). sph_kernel_times returns accumulated milliseconds and
 * launch counts since the last reset: [0] pressure relaxation, [1] density
 * relaxation. */
int sph_set_kernel_timing(sph_handle* h, int32_t enable);
int sph_kernel_times(sph_handle* h, double* ms, int64_t* launches);

/* ---- learned stand-in for the acoustic substeps ------------------------------------ */
/* A message-passing network over the frozen neighbour graph of an advection step that
 * predicts each fluid particle's velocity and density change over the whole step (the
 * paper has no learned component; this is the project's own addition). Definition:
 * node input u_i = [v_i/c0, 100 (rho_i/rho0 - 1), Dt_ad c0/h, 1]; edge input
 * x_ij = [r_ij/h, (v_i - v_j)/c0, 100 dev_i, 100 dev_j, wall] over fluid and wall
 * neighbours (walls: v_j = 0, dev_j = 0); h_i = relu(W_enc u_i); three rounds with shared
 * weights of z_ij = relu(W_e1 [x_ij, h_j, 1]), m_ij = W_e2 [z_ij, 1],
 * a_i = (1/NBAR) sum_j m_ij (NBAR = 20 in 2D, 80 in 3D), h_i += W_n2 [relu(W_n1 [h_i, a_i, 1]), 1];
 * output y_i = W_d2 [relu(W_d1 [h_i, 1]), 1], whose first dim + 1 entries are
 * [(dv_i - g Dt_ad)/V_S, 100 drho_i/rho0] with V_S = |g| Dt_ad (u_ref when g = 0). Every
 * matrix product rounds both operands to
 * bfloat16 and accumulates in FP32 on the tensor cores. Weights: 32,000 floats, matrices
 * enc (64x16), e1 (64x80), e2 (64x80), n1 (64x144), n2 (64x80), d1 (64x80), d2 (16x80),
 * each row-major with inputs zero-padded and the bias in the column after the inputs. */
typedef struct sph_learned sph_learned;

int sph_learned_weight_count(int64_t* count);
/* weights: host or device, 32,000 floats (NULL = zeros). */
int sph_learned_create(int32_t dim, const float* weights, sph_learned** out);
void sph_learned_destroy(sph_learned* net);
const char* sph_learned_last_error(const sph_learned* net);
/* Replace the weights (resets the Adam moments) / read them (host or device pointer). */
int sph_learned_set_weights(sph_learned* net, const float* weights);
int sph_learned_get_weights(sph_learned* net, float* weights);
/* How inference (predict, learned step) runs each round's edge network. enabled = 1 (the
 * default): one fused kernel on warp-level tensor-core MMA; 2: a warp-specialised pipeline
 * on the fifth-generation tensor cores (tcgen05, TMEM accumulators), the node layers then
 * layer by layer; 0: the unfused layers that training uses. All three give bit-identical
 * results. Any other value: SPH_E_INVALID, the setting unchanged. */
int sph_learned_set_fused(sph_learned* net, int32_t enabled);
/* Network output for the handle's current state, which must be the start of an advection
 * step (sph_build_cells then sph_advection_step). y: [n_fluid * (dim+1)] double, id order,
 * host or device (may be NULL). Synchronous. */
int sph_learned_predict(sph_handle* h, sph_learned* net, double* y, void* stream);
/* One training step on the handle's current state (as for predict): forward, mean squared
 * error against target [n_fluid * (dim+1)] (id order, host or device), hand-written
 * backward and, if lr > 0, one Adam step (beta 0.9/0.999, eps 1e-8) on FP32 master
 * weights. loss_out and grad_out (32,000 floats, host or device) may be NULL. */
int sph_learned_train_step(sph_handle* h, sph_learned* net, const double* target, double lr,
                           double* loss_out, float* grad_out, void* stream);
/* One advection step with the network in place of the acoustic substeps: build cells,
 * Dt_ad and density re-initialisation, prediction, then v += g Dt_ad + V_S y_v,
 * rho += rho0 y_rho/100, r += Dt_ad (v + v')/2. If afterwards any tank's mean
 * |rho/rho0 - 1| exceeds max_mean_rho_dev or its energy changed by more than
 * max_energy_drift (relative), the step is undone and the plain acoustic substeps run
 * instead. *used_learned = 1 when the network's step was kept. Synchronous. */
int sph_learned_step(sph_handle* h, sph_learned* net, double max_mean_rho_dev,
                     double max_energy_drift, int32_t* used_learned, void* stream);

/* ---- Species diffusion (Sec. "Schemes for thermal and mass diffusion") ----------------
 * A species C (concentration or temperature) carried by the fluid particles of a handle
 * diffuses by dC/dt = div(D grad C) (Eq. diffusion-eq), discretised as Eq. grad-laplace:
 *   dC_i/dt = 2 sum_j (m_j/rho_j) (C_i - C_j) w(e_ij) (1/r_ij) dW/dr_ij,
 *   w(e) = 1/(L^-1 e)^2 = 1/(e^T D^-1 e),  D = L L^T (Eq. chol),
 * over the fluid neighbours of the current neighbour table (wall particles carry no
 * species: zero flux through walls), with one diffusion tensor D per species object (so
 * the pair combination of the per-particle factors is the factor itself; per-particle
 * multiples of D: sph_species_set_scale) and the masses, densities and positions of the
 * handle's current state. Pairs at zero distance add
 * nothing. Time integration is the two-stage second-order Runge-Kutta scheme (Heun):
 *   C* = C + dt f(C),  C <- (C + C* + dt f(C*)) / 2.
 * For isotropic D = kappa I, w = kappa and the operator is the SPH Laplacian times kappa.
 * For anisotropic D the printed weight is not consistent with div(D grad C) (its
 * continuum limit on a quadratic field differs from tr(D H)); it is computed as printed.
 * The scheme is explicit: dt <= h^2 / (7 lambda_max(D)) is a sufficient stability bound
 * (Gershgorin on the lattice sum of |dW/dr|/r, about 3.5/h^2 in 2D and 3D).
 * The species is stored on the device in FP32, by caller row, so sph_step and
 * sph_build_cells may reorder the particles between diffusion calls. */
typedef struct sph_species sph_species;

/* D: host, dim x dim row-major, symmetric positive definite (else SPH_E_INVALID). The
 * object belongs to handle h (same dimension, particle count) and must be destroyed
 * before it. The species starts at 0. On failure *out may still hold an object that
 * carries the message (sph_species_last_error); destroy it. */
int sph_species_create(sph_handle* h, const double* D, sph_species** out);
void sph_species_destroy(sph_species* sp);
const char* sph_species_last_error(const sph_species* sp);
/* C: host or device, n_fluid doubles in caller row order. Synchronous. */
int sph_species_set(sph_handle* h, sph_species* sp, const double* C, void* stream);
/* C: host or device, n_fluid doubles in caller row order. Synchronous. */
int sph_species_get(sph_handle* h, sph_species* sp, double* C, void* stream);
/* Per-particle diffusivity factors: particle i diffuses with s_i D (s: host or device,
 * n_fluid doubles in caller row order, each positive and finite, else SPH_E_INVALID and
 * no factors). The pair combination of Eq. grad-laplace's per-particle factors, read as
 * the harmonic mean of L~_i = L^-1/sqrt(s_i), weights a pair by
 * ((sqrt(s_i) + sqrt(s_j))/2)^2. Until called, every factor is 1. Synchronous. */
int sph_species_set_scale(sph_handle* h, sph_species* sp, const double* s, void* stream);
/* Per-particle diffusion tensors of different shape: particle i diffuses with D_i (Dp: host
 * or device, n_fluid x dim x dim doubles in caller row order, each row-major, finite,
 * symmetric and positive definite; else SPH_E_INVALID and the species keeps what it had).
 * D_i = L_i L_i^T (Eq. chol); the printed pair combination of the factors, read as the
 * harmonic mean of matrices, weights a pair by r^2 / |M^-1 r|^2, M = (L_i + L_j)/2, which is
 * 1/(e^T D^-1 e) for equal tensors and the sph_species_set_scale weight for D_i = s_i D.
 * Replaces the species' own tensor until called with Dp = NULL; diffusivity factors set by
 * sph_species_set_scale multiply on top (D_i = s_i Dp_i). Synchronous. */
int sph_species_set_tensors(sph_handle* h, sph_species* sp, const double* Dp, void* stream);
/* The kernel-corrected form (Eq. grad-laplace-renormalize) on (on != 0) or off (the
 * default, Eq. grad-laplace). The printed form multiplies the correction matrix B0 by the
 * scalar C; it is taken as the pair weight of Eq. grad-laplace times
 * (e^T B0_i e + e^T B0_j e)/2, which is Eq. grad-laplace for B0 = I, keeps constant fields
 * at rest and conserves the species. B0_i = (sum_j V_j (r_j - r_i) (x) grad_i W_ij)^-1
 * (Eq. sph-correctmatrix) over the species' fluid pairs, V_j = m_j/rho_j, is formed once
 * per sph_diffusion_step call from the current configuration (the identity where that
 * sum is singular: determinant below 1e-6 (trace/d)^d). SPH_E_OOM if its per-particle
 * storage cannot be allocated. Host-only; takes effect at the next diffusion step. */
int sph_species_set_correction(sph_handle* h, sph_species* sp, int32_t on);
/* n_steps RK2 steps of size dt (> 0, finite) on the current neighbour table, which
 * must be valid (sph_build_cells after the last state change; SPH_E_INVALID otherwise).
 * Positions, velocities and densities are not changed. Two kernel launches per step plus
 * a gather and a scatter of the species per call; the call synchronises stream once,
 * after the gather, to learn whether volumes and factors are uniform within each tank
 * (then the stage kernels take them out of the pair loop), and is otherwise
 * asynchronous. */
int sph_diffusion_step(sph_handle* h, sph_species* sp, double dt, int32_t n_steps, void* stream);

/* ---- Reaction step of reaction-diffusion (Sec. "SPH method for reaction-diffusion",
 * "Reaction-by-reaction splitting") ---------------------------------------------------
 * Operator splitting separates the diffusion of the species V (sph_diffusion_step) from the
 * per-particle ODE system dV/dt = I(V, w), dw/dt = g(V, w) (Eq. ode-system) with a gating
 * variable w held by the species object (starts at 0). The caller composes the two, e.g.
 * alternating sph_diffusion_step and sph_reaction_step with the same dt.
 *   model SPH_REACTION_FN, FitzHugh-Nagumo (Eq. fhn):
 *     I = -V (V - a)(V - 1) - w,   g = eps0 (beta V - gamma w - sigma)
 *   model SPH_REACTION_AP, Aliev-Panfilov (Eq. a-p):
 *     I = -k V (V - a)(V - 1) - w V,   g = eps (-k V (V - b - 1) - w),
 *     eps = eps0 + mu1 w / (mu2 + V)
 * One step of length dt applies R_V(dt/2), R_w(dt/2), R_w(dt/2), R_V(dt/2) (Eq.
 * ode-spliting-2rd), each reaction advancing one variable with the other fixed by the
 * quasi-steady-state update y <- y e^(-p dt) + (q/p)(1 - e^(-p dt)) (Eq. ode-qss), with p and
 * q at the reaction's starting value. The split into production q and loss p y:
 *   FN  R_V: q = -w, p = (V - a)(V - 1);        R_w: q = eps0 (beta V - sigma), p = eps0 gamma
 *   AP  R_V: q = 0,  p = k (V - a)(V - 1) + w;  R_w: q = -eps k V (V - b - 1), p = eps
 * (1 - e^(-p dt))/p is taken as dt when |p dt| < 1e-12. Because p and q are frozen over a
 * reaction, the step is first-order accurate where p depends on the reacting variable.
 * Unused parameters of a model are ignored. AP needs mu2 + V != 0 (eps is singular there;
 * the step then produces non-finite values, which the caller sees in sph_species_get).
 * FP32 on the device. */
#define SPH_REACTION_FN 1
#define SPH_REACTION_AP 2
typedef struct {
  int32_t model;                  /* SPH_REACTION_FN or SPH_REACTION_AP */
  double a, b, k, eps0, mu1, mu2, beta, gamma, sigma;
} sph_reaction;

/* w: host or device, n_fluid doubles in caller row order. Synchronous. */
int sph_species_set_gate(sph_handle* h, sph_species* sp, const double* w, void* stream);
/* w: host or device, n_fluid doubles in caller row order. Synchronous. */
int sph_species_get_gate(sph_handle* h, sph_species* sp, double* w, void* stream);
/* n_steps splitting steps of size dt (> 0, finite) of every particle's (V, w), V being the
 * species. No neighbour table needed. Unknown model or non-finite parameters:
 * SPH_E_INVALID. Asynchronous on stream: one kernel launch per call. */
int sph_reaction_step(sph_handle* h, sph_species* sp, const sph_reaction* r, double dt, int32_t n_steps,
                      void* stream);

/* ---- Multi-resolution fluid-structure coupling (Sec. "Multi-resolution FSI coupling") -----
 * An elastic solid with its own particle spacing and smoothing length h_S, attached to a
 * single-tank handle, is coupled to the fluid through the fluid's kernel:
 *  - solid, total Lagrangian (Sec. "Total Lagrangian formulation"): neighbours within 2 h_S in
 *    the reference configuration, kept for the whole run; the true kernel gradient
 *    grad0_a W_ab = dW/dr r0_ab/|r0_ab| and the correction matrix
 *    B0_a = (sum_b V_b (r0_b - r0_a) (x) grad0_a W_ab)^-1 (Eq. sph-correctmatrix), computed once;
 *    first Piola-Kirchhoff stress P = F S, linear elastic S = lambda tr(E) I + 2 mu E or
 *    Neo-Hookean S = mu (I - C^-1) + lambda ln J C^-1 (E = (C - I)/2, C = F^T F, J = det F,
 *    mu = E/(2(1 + nu)), lambda = E nu/((1 + nu)(1 - 2 nu)));
 *    dv_a/dt = (2/m_a) sum_b V_a V_b (P_a B0_a + P_b B0_b)/2 grad0_a W_ab + g + f_a/m_a
 *    (Eq. sph-mechanical-mom), f_a the fluid's force on it;
 *  - solid steps, position-based Verlet (Eqs. verlet-first-half-solid,
 *    verlet-first-mediate-solid, verlet-first-final-solid): F and r half a step, dv/dt, v, r
 *    the second half, dF/dt = (sum_b V_b (v_b - v_a) (x) grad0_a W_ab) B0_a, F the second
 *    half (dF/dt is carried from one step's second half to the next step's first half);
 *  - per fluid acoustic step dt_F: kappa = [dt_F/dt_S] + 1 solid steps of dt_F/kappa, dt_S =
 *    0.6 min(h_S/(c_S + |v|max), sqrt(h_S/|dv/dt|max)) (Eq. dts-advection, c_S = sqrt(K/rho0),
 *    K = lambda + 2 mu/3), with the fluid's force held over them;
 *  - coupling (fluid kernel h_F): after the fluid's pressure relaxation each fluid particle i
 *    near the solid gains sum_a -2 V_i V_a pbar grad_i W(r_ia)/m_i (Eq. fs-force-mr-sp),
 *    pbar = (p_i rho^d + p^d rho_i)/(rho_i + rho^d), the imaginary pressure
 *    p^d = p_i + rho_i max(0, -(g - a~_a).n_a) ((r_i - r_a).n_a) (Eq. fs-coupling-mr read as the
 *    hydrostatic extrapolation along the solid's normal n_a, pointing into the fluid),
 *    rho^d from the EoS, and with viscosity the force of Eq. fs-force-mr-sv with
 *    v^d = 2 v~_a - v_i; the solid takes the opposite forces; after the density relaxation
 *    each such fluid particle adds the continuity term of its solid neighbours as moving
 *    walls (U_L = -n_a.v_i, U_R = -U_L - 2 n_a.v~_a, P_R = p^d). v~_a and a~_a are the solid's
 *    velocity and acceleration averaged over the previous fluid step's solid steps.
 *  Solid particles take no part in the fluid's density re-initialisation. Clamped particles
 *  (fixed[a] != 0) keep their reference position and zero velocity. */
typedef struct sph_solid sph_solid;
#define SPH_SOLID_LINEAR       1
#define SPH_SOLID_NEO_HOOKEAN  2
typedef struct {
  int32_t model;           /* SPH_SOLID_LINEAR or SPH_SOLID_NEO_HOOKEAN                     */
  double  rho0;            /* reference density of the solid                               */
  double  youngs, poisson; /* Young's modulus E > 0 and Poisson ratio -1 < nu < 0.5         */
  double  h;               /* the solid's smoothing length h_S (its support is 2 h_S)      */
  int32_t single_step;     /* 0: multi time stepping (kappa solid steps per fluid acoustic
                              step); 1: single time stepping, the fluid's acoustic step capped
                              at the solid's (kappa = 1 after the first step), the reference
                              the multi-resolution scheme is measured against */
} sph_solid_params;

/* Attach a solid of n particles (1..16384) to a single-tank handle (one solid per handle):
 * pos [n*dim] reference positions inside the handle's cell grid, vol [n] volumes, normal
 * [n*dim] unit normals of the nearest wetted surface (into the fluid), fixed [n] or NULL;
 * host or device arrays, copied. The solid starts undeformed and at rest; the handle's next
 * configuration update (sph_build_cells or a step) includes it, and every later acoustic
 * substep advances it. The κ solid steps of a fluid step run in one thread-block cluster of
 * up to 16 blocks holding the solid in shared memory; internally the particles are kept in
 * a Morton order of their reference positions (outputs come back in the caller's order).
 * Errors: SPH_E_INVALID (arguments, a singular correction matrix), SPH_E_DOMAIN (a particle
 * outside the cell grid), SPH_E_CAPACITY (a reference row longer than the set-up capacity,
 * or a solid that no cluster's shared memory holds), SPH_E_OOM, SPH_E_CUDA. On failure *out
 * may still hold an object carrying the message (sph_solid_last_error); destroy it. */
int sph_solid_create(sph_handle* h, const sph_solid_params* p, int64_t n, const double* pos, const double* vol,
                     const double* normal, const int32_t* fixed, sph_solid** out);
/* Detach from the handle and free; destroy before the handle. */
void sph_solid_destroy(sph_solid* s);
const char* sph_solid_last_error(const sph_solid* s);
/* Number of particles of the solid (the n it was created with), or -1 for NULL: the
 * outputs of sph_solid_get_state hold n*dim (and n*dim*dim) values, dim the handle's. */
int64_t sph_solid_size(const sph_solid* s);
/* The solid's state in the caller's particle order (host or device outputs, any may be
 * NULL): pos, vel, force (the fluid's force held over the last solid steps) [n*dim], F
 * [n*dim*dim] row-major; solid_steps (host) the solid steps taken so far. Synchronous. */
int sph_solid_get_state(sph_handle* h, sph_solid* s, double* pos, double* vel, double* force, double* F,
                        int64_t* solid_steps, void* stream);

/* Allocation-free diagnostics. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory (code running inside
 * another framework's device memory pool or under a fixed device-memory budget,
 * and hosts that forbid runtime allocation after start-up), for whom creating a
 * handle is not an option. It computes the same FP64 fields as sph_diagnostics
 * (t, dt_ad and the step counters are 0) from the caller's arrays in caller order:
 * pos, vel [n*dim], rho, mass [n], all double and all in DEVICE memory of the current
 * device (or managed memory); p supplies
 * dim, rho0, c0 and gravity. out is a host struct; the call synchronises stream.
 * It calls no cudaMalloc, cudaFree or allocating library routine. Its scratch is
 * a fixed 131,200-byte array in the library's device image (1024 blocks of 16
 * partial sums plus the result row), which every GPU that loads the library holds
 * until exit. The first call on each device looks up that array's address with the
 * device current; make that first call before any stream capture begins. Calls
 * share the array and overwrite all of it that they read, so calls that overlap on
 * the GPU race. n above 2^31 - 1, dim not 2 or 3, host pointers, another device's
 * memory or a missing array return SPH_E_INVALID with a message in sph_last_error(NULL);
 * a failed launch returns SPH_E_CUDA (never the previous call's result). The library
 * cannot see array sizes: each array must hold the n (or n*dim) doubles stated. */
int sph_diagnostics_noalloc(const sph_params* p, int64_t n, const double* pos, const double* vel,
                            const double* rho, const double* mass, sph_diag* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_GB300_H */
