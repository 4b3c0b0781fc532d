// Species diffusion on the fluid particles (Sec. "Schemes for thermal and mass diffusion").
//
//   dC_i/dt = 2 sum_j (m_j/rho_j) (C_i - C_j) w(e_ij) (1/r_ij) dW/dr_ij      (Eq. grad-laplace)
//   w(e)    = 1/(L^-1 e)^2 = 1/(e^T D^-1 e),  D = L L^T                        (Eq. chol)
//
// with one diffusion tensor per species object, so the pair combination of the
// per-particle factors is the factor itself; for isotropic D = kappa I, w = kappa.
// Time integration is the two-stage second-order Runge-Kutta scheme (Heun), one kernel
// launch per stage:
//   stage 1: C*      = C^n + dt f(C^n)
//   stage 2: C^{n+1} = (C^n + C* + dt f(C*)) / 2      (written over C^n, own index only)
//
// One thread per fluid particle walks the fluid part of its neighbour row in the
// quad-interleaved table, keeping the next index quad in flight, and gathers per neighbour
// the 16-byte position record (fixed-point position + density deviation, the same record
// the relaxations read) and the 4-byte species value. Pair vectors are exact integer
// differences scaled by the position quantum. Wall neighbours are skipped: walls carry no
// species (zero flux). Pairs at zero distance add nothing.
//
// Between calls the species is kept by caller row, so the fluid solver may re-sort the
// particles; each call gathers it into slot order, runs its steps and scatters it back.
#include <cmath>
#include <string>
#include <vector>

#include "sph_handle.h"

namespace sph {
namespace {

constexpr int kDiffBlock = 256;

// Symmetric D^-1 (xx, yy, zz, xy, xz, yz) and the isotropic coefficient.
struct DiffCoef {
  float xx, yy, zz, xy, xz, yz, kappa;
};

inline unsigned diff_grid(int64_t n) { return (unsigned)((n + kDiffBlock - 1) / kDiffBlock); }

template <bool PER>
__device__ __forceinline__ float axis_diff(int qi, int qj, int period, float dq) {
  return (float)(PER ? wrap_diff(qi - qj, period) : qi - qj) * dq;
}

// One pair's share of f(C)_i / 2, zero at zero distance and beyond 2h.
template <int D, bool PER, bool ISO>
__device__ __forceinline__ float diff_term(const Inst& I, const DiffCoef& K, const int4& pi, float ci,
                                           const int4& a, float ca, float ma) {
  const float rx = axis_diff<PER>(pi.x, a.x, I.period[0], I.dq);
  const float ry = axis_diff<PER>(pi.y, a.y, I.period[1], I.dq);
  const float rz = D == 3 ? axis_diff<PER>(pi.z, a.z, I.period[2], I.dq) : 0.0f;
  const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
  const float r = r2 * rsqrtf(r2);
  const float t = fmaxf(fmaf(r, -0.5f * I.inv_h, 1.0f), 0.0f);
  const float fw = I.dwr_a * (t * t * t);                         // (dW/dr)/r, Wendland C2
  float w;
  if (ISO) {
    w = K.kappa;
  } else {
    float qf = fmaf(K.xx * rx, rx, fmaf(K.yy * ry, ry, 2.0f * K.xy * rx * ry));
    if (D == 3) qf = fmaf(K.zz * rz, rz, fmaf(2.0f * K.xz * rx, rz, fmaf(2.0f * K.yz * ry, rz, qf)));
    w = __fdividef(r2, qf);                                        // 1/(e^T D^-1 e)
  }
  const float vj = __fdividef(ma, I.rho0 + i2f(a.w));              // m_j / rho_j
  const float term = vj * (ci - ca) * fw * w;
  return r2 > 0.0f ? term : 0.0f;
}

template <int D, bool PER, bool ISO, bool SECOND>
__global__ void __launch_bounds__(kDiffBlock)
k_diffusion_stage(int64_t n, const int4* __restrict__ P, const float* __restrict__ Cin, const float* Cn,
                  float* Cout, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                  const int* __restrict__ inst_of, const Inst* __restrict__ inst,
                  const float* __restrict__ mass, DiffCoef K, float dt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const int4 pi = P[i];
  const float ci = Cin[i];
  const int nf = (int)(nbc[i] & 0xffffu);
  const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
  const int nq = (nf + 3) >> 2;
  float s0 = 0.0f, s1 = 0.0f;
  int4 nxt = nq ? nb4[i] : make_int4(0, 0, 0, 0);
  for (int q = 0; q < nq; ++q) {
    const int4 cq = nxt;
    if (q + 1 < nq) nxt = nb4[(int64_t)(q + 1) * n + i];   // next quad in flight
    const int sl = q << 2;
    const int j1 = sl + 1 < nf ? cq.y : cq.x, j2 = sl + 2 < nf ? cq.z : cq.x, j3 = sl + 3 < nf ? cq.w : cq.x;
    const int4 a0 = P[cq.x], a1 = P[j1], a2 = P[j2], a3 = P[j3];
    const float c0 = Cin[cq.x], c1 = Cin[j1], c2 = Cin[j2], c3 = Cin[j3];
    float m0 = I.mass, m1 = I.mass, m2 = I.mass, m3 = I.mass;
    if (mass) {
      m0 = mass[cq.x]; m1 = mass[j1]; m2 = mass[j2]; m3 = mass[j3];
    }
    s0 += diff_term<D, PER, ISO>(I, K, pi, ci, a0, c0, m0);
    const float t1 = diff_term<D, PER, ISO>(I, K, pi, ci, a1, c1, m1);
    const float t2 = diff_term<D, PER, ISO>(I, K, pi, ci, a2, c2, m2);
    const float t3 = diff_term<D, PER, ISO>(I, K, pi, ci, a3, c3, m3);
    s1 += sl + 1 < nf ? t1 : 0.0f;
    s0 += sl + 2 < nf ? t2 : 0.0f;
    s1 += sl + 3 < nf ? t3 : 0.0f;
  }
  const float rate = 2.0f * (s0 + s1);
  const float next = fmaf(dt, rate, ci);
  Cout[i] = SECOND ? 0.5f * (Cn[i] + next) : next;
}

// Caller row -> slot order and back (b.id[slot] = caller row).
__global__ void k_species_gather(int64_t n, const int* __restrict__ id, const float* __restrict__ by_row,
                                 float* __restrict__ by_slot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) by_slot[i] = by_row[id[i]];
}

__global__ void k_species_scatter(int64_t n, const int* __restrict__ id, const float* __restrict__ by_slot,
                                  float* __restrict__ by_row) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) by_row[id[i]] = by_slot[i];
}

__global__ void k_species_import(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

__global__ void k_species_export(int64_t n, const float* __restrict__ src, double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

using StageFn = void (*)(int64_t, const int4*, const float*, const float*, float*, const int*,
                         const uint32_t*, const int*, const Inst*, const float*, DiffCoef, float);

template <int D, bool PER, bool ISO>
void pick_stages(StageFn* s1, StageFn* s2) {
  *s1 = k_diffusion_stage<D, PER, ISO, false>;
  *s2 = k_diffusion_stage<D, PER, ISO, true>;
}

template <int D, bool PER>
void pick_stages(bool iso, StageFn* s1, StageFn* s2) {
  if (iso) pick_stages<D, PER, true>(s1, s2);
  else pick_stages<D, PER, false>(s1, s2);
}

}  // namespace
}  // namespace sph

struct sph_species {
  int dim = 0;
  int64_t n = 0;
  sph::DiffCoef K{};
  bool iso = false;
  float* by_row = nullptr;     // [n] species by caller row (kept between calls)
  float* ca = nullptr;         // [n] slot order: C^n
  float* cb = nullptr;         // [n] slot order: C*
  double* stage = nullptr;     // [n] doubles for host copies
  std::string err;
};

namespace {

int sfail(sph_species* sp, int code, const std::string& msg) {
  if (sp) sp->err = msg;
  return code;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Cholesky factor of a symmetric d x d tensor (row-major); false unless positive definite.
bool cholesky(const double* D, int d, double* L) {
  for (int k = 0; k < 9; ++k) L[k] = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = D[i * d + j];
      for (int k = 0; k < j; ++k) s -= L[i * 3 + k] * L[j * 3 + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i * 3 + i] = std::sqrt(s);
      } else {
        L[i * 3 + j] = s / L[j * 3 + j];
      }
    }
  return true;
}

// D^-1 = L^-T L^-1 from the lower-triangular factor (3 x 3 storage).
void inverse_from_cholesky(const double* L, int d, double* Dinv) {
  double Li[9] = {0};
  for (int i = 0; i < d; ++i) {
    Li[i * 3 + i] = 1.0 / L[i * 3 + i];
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s -= L[i * 3 + k] * Li[k * 3 + j];
      Li[i * 3 + j] = s / L[i * 3 + i];
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += Li[k * 3 + a] * Li[k * 3 + b];
      Dinv[a * 3 + b] = s;
    }
}

}  // namespace

extern "C" {

int sph_species_create(sph_handle* h, const double* D, sph_species** out) {
  if (!out) return SPH_E_INVALID;
  *out = nullptr;
  if (!h || !D) return SPH_E_INVALID;
  auto* sp = new sph_species();
  *out = sp;
  const int d = h->b.dim;
  sp->dim = d;
  sp->n = h->b.n;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (!std::isfinite(D[i * d + j]) || D[i * d + j] != D[j * d + i])
        return sfail(sp, SPH_E_INVALID, "D must be finite and symmetric");
  double L[9], Dinv[9];
  if (!cholesky(D, d, L)) return sfail(sp, SPH_E_INVALID, "D must be positive definite");
  inverse_from_cholesky(L, d, Dinv);
  bool iso = true;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (D[i * d + j] != (i == j ? D[0] : 0.0)) iso = false;
  sp->iso = iso;
  sp->K = sph::DiffCoef{(float)Dinv[0], (float)Dinv[4], (float)Dinv[8], (float)Dinv[1],
                        (float)Dinv[2], (float)Dinv[5], (float)D[0]};
  if (sp->n > 0) {
    const size_t n = (size_t)sp->n;
    if (cudaMalloc(&sp->by_row, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&sp->ca, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&sp->cb, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&sp->stage, sizeof(double) * n) != cudaSuccess) {
      cudaGetLastError();
      return sfail(sp, SPH_E_OOM, "device allocation of the species failed");
    }
    if (cudaMemset(sp->by_row, 0, sizeof(float) * n) != cudaSuccess)
      return sfail(sp, SPH_E_CUDA, "clearing the species failed");
  }
  return SPH_OK;
}

void sph_species_destroy(sph_species* sp) {
  if (!sp) return;
  cudaFree(sp->by_row);
  cudaFree(sp->ca);
  cudaFree(sp->cb);
  cudaFree(sp->stage);
  delete sp;
}

const char* sph_species_last_error(const sph_species* sp) { return sp ? sp->err.c_str() : "null species"; }

int sph_species_set(sph_handle* h, sph_species* sp, const double* C, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (sp->n == 0) return SPH_OK;
  if (!C) return sfail(sp, SPH_E_INVALID, "C is required");
  cudaStream_t s = (cudaStream_t)stream;
  const double* src = C;
  if (!device_pointer(C)) {
    if (cudaMemcpyAsync(sp->stage, C, sizeof(double) * sp->n, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return sfail(sp, SPH_E_CUDA, "copy of the species failed");
    src = sp->stage;
  }
  sph::k_species_import<<<sph::diff_grid(sp->n), sph::kDiffBlock, 0, s>>>(sp->n, src, sp->by_row);
  ++h->launches;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "species upload failed");
  return SPH_OK;
}

int sph_species_get(sph_handle* h, sph_species* sp, double* C, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (sp->n == 0) return SPH_OK;
  if (!C) return sfail(sp, SPH_E_INVALID, "C is required");
  cudaStream_t s = (cudaStream_t)stream;
  const bool dev = device_pointer(C);
  double* dst = dev ? C : sp->stage;
  sph::k_species_export<<<sph::diff_grid(sp->n), sph::kDiffBlock, 0, s>>>(sp->n, sp->by_row, dst);
  ++h->launches;
  if (!dev && cudaMemcpyAsync(C, sp->stage, sizeof(double) * sp->n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "copy of the species failed");
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return sfail(sp, SPH_E_CUDA, "species download failed");
  return SPH_OK;
}

int sph_diffusion_step(sph_handle* h, sph_species* sp, double dt, int32_t n_steps, void* stream) {
  if (!h || !sp) return SPH_E_INVALID;
  if (sp->n != h->b.n || sp->dim != h->b.dim) return sfail(sp, SPH_E_INVALID, "species belongs to another handle");
  if (!(std::isfinite(dt) && dt > 0.0) || n_steps < 0) return sfail(sp, SPH_E_INVALID, "dt must be > 0 and n_steps >= 0");
  if (!h->cells_valid) return sfail(sp, SPH_E_INVALID, "sph_build_cells must run after a state change");
  const sph::Buffers& b = h->b;
  if (b.n == 0 || n_steps == 0) return SPH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  sph::StageFn s1, s2;
  if (b.dim == 2) {
    if (b.any_periodic) sph::pick_stages<2, true>(sp->iso, &s1, &s2);
    else sph::pick_stages<2, false>(sp->iso, &s1, &s2);
  } else {
    if (b.any_periodic) sph::pick_stages<3, true>(sp->iso, &s1, &s2);
    else sph::pick_stages<3, false>(sp->iso, &s1, &s2);
  }
  const unsigned grid = sph::diff_grid(b.n);
  const float fdt = (float)dt;
  sph::k_species_gather<<<grid, sph::kDiffBlock, 0, s>>>(b.n, b.id, sp->by_row, sp->ca);
  for (int k = 0; k < n_steps; ++k) {
    s1<<<grid, sph::kDiffBlock, 0, s>>>(b.n, b.PS, sp->ca, nullptr, sp->cb, b.nbr, b.nbc, b.inst_of,
                                         b.inst, b.mass, sp->K, fdt);
    s2<<<grid, sph::kDiffBlock, 0, s>>>(b.n, b.PS, sp->cb, sp->ca, sp->ca, b.nbr, b.nbc, b.inst_of,
                                         b.inst, b.mass, sp->K, fdt);
  }
  sph::k_species_scatter<<<grid, sph::kDiffBlock, 0, s>>>(b.n, b.id, sp->ca, sp->by_row);
  h->launches += 2 + 2 * (int64_t)n_steps;
  if (cudaGetLastError() != cudaSuccess) return sfail(sp, SPH_E_CUDA, "diffusion launch failed");
  return SPH_OK;
}

}  // extern "C"
