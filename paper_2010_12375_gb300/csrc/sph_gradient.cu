// Particle gradients of the density and the pressure (paper Sec. 1.1, "particle average
// and gradient"): the strong form of Eq. gradsph-strong, which determines the local
// structure of a field, and the weak form of Eq. gradsph-weak, which conserves.
//
// The paper writes both with grad_i W_ij = e_ij dW/dr, e_ij pointing from i to j, which is
// minus the true gradient; with the true gradient grad_i W_ij = (dW/dr) r_ij / |r_ij|,
// r_ij = r_i - r_j, they read
//   strong  grad f_i = sum_j V_j (f_j - f_i) grad_i W_ij
//   weak    grad f_i = sum_j V_j (f_i + f_j) grad_i W_ij
// over the fluid neighbours (V_j = m_j / rho_j) and the wall neighbours, which carry the
// values of the one-sided wall problem: p_w = p_i + rho_i g.(r_w - r_i), rho_w = rho0 + p_w/c0^2,
// volume V_w.
//
// With the linear EoS p = c0^2 (rho - rho0) all four fields follow from three vector sums
// per particle (dev = rho - rho0, delta_w = rho_i g.(r_w - r_i) / c0^2 = rho_w - rho_i):
//   S  = sum V grad_i W                          (fluid and wall pairs)
//   As = sum_fluid V (dev_j - dev_i) grad + sum_wall V delta_w grad
//   Aw = sum_fluid V (dev_i + dev_j) grad + sum_wall V (2 dev_i + delta_w) grad
//   grad rho: strong As, weak Aw + 2 rho0 S;   grad p: strong c0^2 As, weak c0^2 Aw.
// Writing rho_i + rho_j as 2 rho0 + dev_i + dev_j keeps the large, cancelling 2 rho0 part in
// S, summed on its own. One thread per fluid particle walks its row of the current
// neighbour table with the pair geometry from the current positions (as the relaxations
// do); every sum is Kahan-compensated in FP32.
#include "sph.h"
#include "sph_handle.h"
#include "sph_kernels.h"

namespace sph {
namespace {

constexpr int kGradBlock = 128;

struct Kahan3 {
  float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void add(float w, float rx, float ry, float rz) {
    const float v[3] = {w * rx, w * ry, w * rz};
#pragma unroll
    for (int a = 0; a < 3; ++a) kahan_add(s[a], c[a], v[a]);
  }
};

template <bool PER>
__device__ __forceinline__ float exact_axis(int qi, int qj, int period, float dq) {
  return (biased_diff<PER>(qi, qj, period) - kMagic) * dq;
}

template <int D, bool PER>
__global__ void __launch_bounds__(kGradBlock)
k_gradients(int64_t n, const int4* __restrict__ PS, const float* __restrict__ mass, const int* __restrict__ inst_of,
            const Inst* __restrict__ inst, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
            const int4* __restrict__ WP, float4* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const int4 pi = PS[i];
  const float dev_i = i2f(pi.w);
  const float rho_i = I.rho0 + dev_i;
  const int px = PER ? I.period[0] : 0, py = PER ? I.period[1] : 0, pz = PER ? I.period[2] : 0;
  const uint32_t cnt = nbc[i];
  const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
  Kahan3 S, As, Aw;
  for (int s = 0; s < nf; ++s) {
    const int j = nbr[slot_index(n, i, s)];
    const int4 pj = PS[j];
    const float rx = exact_axis<PER>(pi.x, pj.x, px, I.dq);
    const float ry = exact_axis<PER>(pi.y, pj.y, py, I.dq);
    const float rz = D == 3 ? exact_axis<PER>(pi.z, pj.z, pz, I.dq) : 0.f;
    const float r = sqrtf(rx * rx + ry * ry + rz * rz);
    const float dev_j = i2f(pj.w);
    const float Vj = (mass ? mass[j] : I.mass) / (I.rho0 + dev_j);
    const float w = Vj * kernel_dW_over_r(r, I);            // V_j (dW/dr)/r; r_ij below
    S.add(w, rx, ry, rz);
    As.add(w * (dev_j - dev_i), rx, ry, rz);
    Aw.add(w * (dev_i + dev_j), rx, ry, rz);
  }
  const int w0 = wall_slot0(nf);
  for (int s = 0; s < nw; ++s) {
    const int k = nbr[slot_index(n, i, w0 + s)];
    const int4 qw = WP[k];
    const float rx = exact_axis<PER>(pi.x, qw.x, px, I.dq);
    const float ry = exact_axis<PER>(pi.y, qw.y, py, I.dq);
    const float rz = D == 3 ? exact_axis<PER>(pi.z, qw.z, pz, I.dq) : 0.f;
    const float r = sqrtf(rx * rx + ry * ry + rz * rz);
    // rho_w - rho_i = rho_i g.(r_w - r_i) / c0^2, and r_w - r_i = -r_iw
    const float delta = -rho_i * (I.g[0] * rx + I.g[1] * ry + I.g[2] * rz) * I.inv_c0sq;
    const float w = i2f(qw.w) * kernel_dW_over_r(r, I);
    S.add(w, rx, ry, rz);
    As.add(w * delta, rx, ry, rz);
    Aw.add(w * (2.0f * dev_i + delta), rx, ry, rz);
  }
  auto total = [](const Kahan3& k, int a) { return k.s[a] - k.c[a]; };
  out[i] = make_float4(total(As, 0), total(As, 1), total(As, 2), 0.f);
  out[n + i] = make_float4(total(Aw, 0), total(Aw, 1), total(Aw, 2), 0.f);
  out[2 * n + i] = make_float4(total(S, 0), total(S, 1), total(S, 2), 0.f);
}

// which: 0 grad rho strong, 1 grad rho weak, 2 grad p strong, 3 grad p weak; caller row order
__global__ void k_export_gradient(int64_t n, int dim, int which, const float4* __restrict__ G,
                                  const int* __restrict__ id, const int* __restrict__ inst_of,
                                  const Inst* __restrict__ inst, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const double c0sq = I.c0_d * I.c0_d;
  const float4 As = G[i], Aw = G[n + i], S = G[2 * n + i];
  const double as[3] = {As.x, As.y, As.z}, aw[3] = {Aw.x, Aw.y, Aw.z}, sv[3] = {S.x, S.y, S.z};
  const int64_t row = id[i];
  for (int a = 0; a < dim; ++a) {
    double v;
    if (which == 0) v = as[a];
    else if (which == 1) v = aw[a] + 2.0 * I.rho0_d * sv[a];
    else if (which == 2) v = c0sq * as[a];
    else v = c0sq * aw[a];
    out[row * dim + a] = v;
  }
}

}  // namespace
}  // namespace sph

namespace {

bool addressable(const void* p) {       // memory the current device writes directly
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
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

bool other_device(const void* p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int cur = -1;
  if (at.type != cudaMemoryTypeDevice || cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.device != cur;
}

int gfail(sph_handle* h, int code, const char* msg) {
  h->err = msg;
  return code;
}

}  // namespace

extern "C" int sph_gradient_diagnostics(sph_handle* h, double* grad_rho_strong, double* grad_rho_weak,
                                        double* grad_p_strong, double* grad_p_weak, void* stream) {
  if (!h) return SPH_E_INVALID;
  double* outs[4] = {grad_rho_strong, grad_rho_weak, grad_p_strong, grad_p_weak};
  for (double* o : outs)
    if (other_device(o)) return gfail(h, SPH_E_INVALID, "an output array lives on another device");
  if (!h->cells_valid) return gfail(h, SPH_E_INVALID, "sph_build_cells must run after a state change");
  cudaStream_t s = (cudaStream_t)stream;
  const sph::Buffers& b = h->b;
  if (b.n == 0) return SPH_OK;
  int r = sph_debug_check(h, s);
  if (r != SPH_OK) return r;
  if (!h->grad) {
    if (cudaMalloc(&h->grad, sizeof(float4) * 3 * (size_t)b.n) != cudaSuccess) {
      cudaGetLastError();
      h->grad = nullptr;
      return gfail(h, SPH_E_OOM, "device allocation of the gradient buffer failed");
    }
    h->allocs.push_back(h->grad);
    h->device_bytes += (int64_t)(sizeof(float4) * 3 * (size_t)b.n);
  }
  const unsigned grid = (unsigned)((b.n + sph::kGradBlock - 1) / sph::kGradBlock);
  auto kern = b.dim == 2 ? (b.any_periodic ? sph::k_gradients<2, true> : sph::k_gradients<2, false>)
                         : (b.any_periodic ? sph::k_gradients<3, true> : sph::k_gradients<3, false>);
  kern<<<grid, sph::kGradBlock, 0, s>>>(b.n, b.PS, b.mass, b.inst_of, b.inst, b.nbr, b.nbc, b.nw ? b.WP : nullptr,
                                        h->grad);
  ++h->launches;
  const size_t elems = (size_t)b.n * b.dim;
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    const bool dev = addressable(outs[k]);
    double* tgt = dev ? outs[k] : h->stage;            // the stage holds >= n * dim doubles
    sph::k_export_gradient<<<grid, sph::kGradBlock, 0, s>>>(b.n, b.dim, k, h->grad, b.id, b.inst_of, b.inst, tgt);
    ++h->launches;
    if (!dev && cudaMemcpyAsync(outs[k], tgt, sizeof(double) * elems, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      cudaGetLastError();
      return gfail(h, SPH_E_CUDA, "copy of a gradient failed");
    }
  }
  if (cudaGetLastError() != cudaSuccess) return gfail(h, SPH_E_CUDA, "gradient launch failed");
  return sph_sync_status(h, s);
}
