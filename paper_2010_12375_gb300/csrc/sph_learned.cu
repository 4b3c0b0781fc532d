// Learned stand-in for the acoustic substeps of an advection step.
//
// A message-passing network over the frozen neighbour graph of the step predicts each
// fluid particle's velocity and density change over Dt_ad (the network is the project's
// own; the paper has none). Definition (an FP64 reference implementation of the same
// network is kept with the tests):
//   u_i  = [v_i/c0, 100 (rho_i/rho0 - 1), Dt_ad c0/h, 1]                      K = 16
//   x_ij = [r_ij/h, (v_i - v_j)/c0, 100 dev_i, 100 dev_j, wall]  (walls: v_j = 0, dev_j = 0)
//   h_i  = relu(W_enc u_i)
//   3 rounds, shared weights:
//     z_ij = relu(W_e1 [x_ij, h_j, 1])     m_ij = W_e2 [z_ij, 1]            K = 80, 80
//     a_i  = (1/NBAR) sum_j m_ij           h_i += W_n2 [relu(W_n1 [h_i, a_i, 1]), 1]   K = 144, 80
//   y_i  = W_d2 [relu(W_d1 [h_i, 1]), 1]                                     K = 80, 80
//   targets [(dv_i - g Dt_ad)/V_S, 100 drho_i/rho0], V_S = |g| Dt_ad (U_ref when g = 0),
//   loss = mean squared error.
// Every product rounds its operands to bfloat16 and accumulates in FP32 on the tensor
// cores: the layer-by-layer path (training, and inference when the fused rounds are off)
// on the fifth-generation tensor cores (tcgen05, 128-row tiles, accumulators in TMEM; see
// sph_tc.cuh), the fused inference rounds with warp-level mma.sync m16n8k16 (both sum each
// 16-wide K step in the same order, so the two paths agree bit for bit). These layers are
// skinny (64 outputs, K <= 144: ~34 FLOP per byte moved, far below the tensor-core ridge of
// ~285), so unfused they are bound by HBM, not by the MMA. Weight gradients are summed per block and then over
// blocks in a fixed order and node-embedding gradients of the neighbour gather are summed
// per node over its reverse edges in edge order, so a training step is deterministic (only
// the reported loss value is accumulated with atomics).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sph.h"
#include "sph_handle.h"
#include "sph_kernels.h"
#include "sph_tc.cuh"

using bf16 = __nv_bfloat16;

namespace sph {
namespace learned {

constexpr int F = 64;
constexpr int ROUNDS = 3;
constexpr float S_RHO = 100.0f;
enum { L_ENC = 0, L_E1, L_E2, L_N1, L_N2, L_D1, L_D2, L_COUNT };
constexpr int kRows[L_COUNT] = {64, 64, 64, 64, 64, 64, 16};
constexpr int kCols[L_COUNT] = {16, 80, 80, 144, 80, 80, 80};
__constant__ int c_rows[L_COUNT] = {64, 64, 64, 64, 64, 64, 16};
__constant__ int c_cols[L_COUNT] = {16, 80, 80, 144, 80, 80, 80};
constexpr int kWeights = 32000;
constexpr int kTile = 64;                 // rows per dense block (4 warps x 16)
constexpr int kDwRows = 2048;             // rows per weight-gradient block

inline int w_offset(int l) {
  int o = 0;
  for (int k = 0; k < l; ++k) o += kRows[k] * kCols[k];
  return o;
}

inline float nbar(int dim) { return dim == 2 ? 20.0f : 80.0f; }

__device__ __forceinline__ uint32_t ld_u32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------------ dense forward
// Y = X W^T for M rows on the fifth-generation tensor cores (sph_tc.cuh). Each CTA (one
// warpgroup of 128 threads) keeps W [NO x K] in shared memory in the core-matrix layout and
// walks 128-row tiles (grid-stride): the tile's rows are copied into the A operand, one
// thread issues the K/16 MMAs into TMEM, and each warp then reads its 32 rows' accumulators
// (TMEM lane = row) 16 columns at a time for the epilogue. Epilogue per element
// (m, n < NO): y = acc; y = 0 where mask[m, n] <= 0 (ReLU backward) if mask;
// y = max(y, 0) if relu; out_f32[m, n] = y (or += y with accum) for n < nf_store;
// out_b[m, col0 + n] = bf16(y) for n < nb_store. Copies are shaped for the memory system:
// a quarter-warp moves one core matrix (8 rows x 16 bytes: one 128-byte shared-memory
// wavefront, two full global sectors per row pair of pieces), and each warp stages its
// 32 x 16 block of results in shared memory (in the tile the tensor core has just read, so
// the staging costs no shared memory of its own) to store them as 64-byte row segments.
// K is a multiple of 16, ldx, ldo, col0 and nb_store multiples of 8, ldf and nf_store of 4,
// ldm of 2 (checked by the host wrapper). A wait for the tensor core that runs out sets
// ERR_TIMEOUT in *err and the CTA stops.
constexpr int kDenseStageLd = 17;           // staged row stride (floats): conflict-free columns

// shared memory of k_dense: W, then two row tiles of 128 x K, each large enough to serve as
// the four warps' staging blocks once the tensor core has read it
__host__ __device__ constexpr int dense_w_bytes(int NO, int K) { return (NO * K * 2 + 127) / 128 * 128; }
__host__ __device__ constexpr int dense_tile_bytes(int K) {
  return ((128 * K * 2 > 4 * 32 * kDenseStageLd * 4 ? 128 * K * 2 : 4 * 32 * kDenseStageLd * 4) + 127) / 128 * 128;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;                       // 0: fill the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// 16-byte pieces of an R-row operand, [R x K] row-major in global memory (row stride ld
// elements), into the core-matrix layout: piece (row, kc) by lane (row % 8) + 8 (kc % 4) of a
// warp-sized block of 8 rows x 4 pieces. Rows at or past rows_valid are zero. ASYNC: by
// cp.async (zero-filled past rows_valid), completed by the caller's cp_async_wait_all.
template <bool ASYNC>
__device__ __forceinline__ void load_operand(unsigned char* dst, int R, int K, const bf16* __restrict__ src,
                                             int64_t ld, int64_t rows_valid) {
  const int KC = K / 8, KB = (KC + 3) / 4;           // pieces per row, 4-piece groups
  const int blocks = (R / 8) * KB;
  const int lane = threadIdx.x & 31;
  for (int blk = threadIdx.x >> 5; blk < blocks; blk += blockDim.x >> 5) {
    const int r = (blk / KB) * 8 + (lane & 7), kc = (blk % KB) * 4 + (lane >> 3);
    if (kc >= KC) continue;
    const bool valid = r < rows_valid;
    unsigned char* d = dst + tc::core_offset(R, r, kc * 8);
    if (ASYNC) {
      cp_async16(d, src + (valid ? (int64_t)r * ld : 0) + kc * 8, valid);
    } else {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (valid) v = *reinterpret_cast<const uint4*>(src + (int64_t)r * ld + kc * 8);
      *reinterpret_cast<uint4*>(d) = v;
    }
  }
}

template <int NO>
__global__ void __launch_bounds__(128)
k_dense(int64_t M, int K, const bf16* __restrict__ X, int ldx, const bf16* __restrict__ W,
        float* __restrict__ out_f32, int ldf, int nf_store, int accum, bf16* __restrict__ out_b, int ldo,
        int col0, int nb_store, int relu, const bf16* __restrict__ mask, int ldm, int* __restrict__ err) {
  constexpr int COLS = tc::tmem_cols(NO);
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  unsigned char* sB = tc_smem;                        // NO x K
  const int tile_bytes = dense_tile_bytes(K);
  unsigned char* sA0 = tc_smem + dense_w_bytes(NO, K);   // two 128 x K row tiles
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_operand<false>(sB, NO, K, W, K, NO);
  if (threadIdx.x == 0) tc::mbar_init(&bar);
  if (warp == 0) tc::tmem_alloc(&tmem_slot, COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t b_addr = tc::smem_u32(sB);
  const int64_t tiles = (M + 127) / 128;
  uint32_t phase = 0;
  if (blockIdx.x < tiles) {                           // the first tile streams in
    const int64_t m0 = (int64_t)blockIdx.x * 128;
    load_operand<true>(sA0, 128, K, X + m0 * ldx, ldx, M - m0);
  }
  cp_async_commit();
  int buf = 0;
  float* st = nullptr;                                // this warp's staging block, in the tile just multiplied
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, buf ^= 1) {
    const int64_t m0 = tile * 128;
    unsigned char* sA = sA0 + buf * tile_bytes;
    cp_async_wait_all();
    tc::fence_to_async();
    __syncthreads();                                  // this tile in place; the other buffer free
    const int64_t next = tile + gridDim.x;
    if (next < tiles)                                 // the next tile streams in meanwhile
      load_operand<true>(sA0 + (buf ^ 1) * tile_bytes, 128, K, X + next * 128 * ldx, ldx, M - next * 128);
    cp_async_commit();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      tc::mma_tile<NO>(tmem, tc::smem_u32(sA), b_addr, K, false, &bar);
    }
    const bool done = tc::mbar_wait(&bar, phase);
    phase ^= 1u;
    if (!__syncthreads_and(done)) {                   // the same decision in every thread
      if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
      break;
    }
    tc::fence_after_sync();
    st = reinterpret_cast<float*>(sA) + warp * 32 * kDenseStageLd;   // the tensor core is done with the tile
    const int64_t mw = m0 + warp * 32;                // this warp's first row
    const int64_t my = mw + lane;                     // the row whose accumulators this lane reads
#pragma unroll 1
    for (int c0 = 0; c0 < NO; c0 += 16) {
      float y[16];
      tc::tmem_ld16(tc::tmem_addr(tmem, warp, c0), y);
      if (mask && my < M) {
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          const uint32_t mk = ld_u32(&mask[my * ldm + c0 + q]);
          if (!(__bfloat162float(__ushort_as_bfloat16((unsigned short)(mk & 0xffffu))) > 0.f)) y[q] = 0.f;
          if (!(__bfloat162float(__ushort_as_bfloat16((unsigned short)(mk >> 16))) > 0.f)) y[q + 1] = 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) st[lane * kDenseStageLd + q] = relu ? fmaxf(y[q], 0.f) : y[q];
      __syncwarp();
      if (out_f32 && c0 < nf_store) {                 // 8 rows x 4 float4 pieces per pass
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
          const int r = pass * 8 + (lane >> 2), c = (lane & 3) * 4;
          const int64_t m = mw + r;
          if (m < M && c0 + c < nf_store) {
            const float* v = st + r * kDenseStageLd + c;
            float4 o = make_float4(v[0], v[1], v[2], v[3]);
            float4* dst = reinterpret_cast<float4*>(&out_f32[m * ldf + c0 + c]);
            if (accum) {
              const float4 p = *dst;
              o = make_float4(p.x + o.x, p.y + o.y, p.z + o.z, p.w + o.w);
            }
            *dst = o;
          }
        }
      }
      if (out_b && c0 < nb_store) {                   // 16 rows x 2 pieces of 8 bf16 per pass
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const int r = pass * 16 + (lane >> 1), c = (lane & 1) * 8;
          const int64_t m = mw + r;
          if (m < M && c0 + c < nb_store) {
            const float* v = st + r * kDenseStageLd + c;
            uint4 o;
            o.x = pack2(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
            o.y = pack2(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
            o.z = pack2(__float2bfloat16_rn(v[4]), __float2bfloat16_rn(v[5]));
            o.w = pack2(__float2bfloat16_rn(v[6]), __float2bfloat16_rn(v[7]));
            *reinterpret_cast<uint4*>(&out_b[m * ldo + col0 + c0 + c]) = o;
          }
        }
      }
      __syncwarp();                                   // the staging block is reused next
    }
    tc::fence_before_sync();
    __syncthreads();                                  // TMEM read and the A tile free before the next
  }
  cp_async_wait_all();                                // no copy left in flight at exit
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, COLS);
}

// ------------------------------------------------------------------ weight gradient
// partial[block][no][k] = sum over this block's rows m of dY[m, no] X[m, k] (tensor cores,
// the row index is the MMA reduction dimension).
template <int NO>
__global__ void __launch_bounds__(128)
k_dense_dw(int64_t M, int K, const bf16* __restrict__ dY, int ldy, const bf16* __restrict__ X, int ldx,
           float* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LDY = NO + 8, LDX = K + 8;
  bf16* sY = reinterpret_cast<bf16*>(smem_raw);
  bf16* sX = sY + kTile * LDY;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt_n = NO / 16, nt_n = K / 8, tiles = mt_n * nt_n;
  constexpr int kMaxT = (NO / 16) * 18 / 4 + 1;   // K <= 144 -> at most 18 column tiles
  float acc[kMaxT][4];
#pragma unroll
  for (int q = 0; q < kMaxT; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
  const int64_t r_begin = (int64_t)blockIdx.x * kDwRows;
  const int64_t r_end = min(r_begin + (int64_t)kDwRows, M);
  for (int64_t c0 = r_begin; c0 < r_end; c0 += kTile) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTile * NO; idx += blockDim.x) {
      const int r = idx / NO, c = idx % NO;
      const int64_t m = c0 + r;
      sY[r * LDY + c] = m < r_end ? dY[m * ldy + c] : __float2bfloat16_rn(0.f);
    }
    for (int idx = threadIdx.x; idx < kTile * K; idx += blockDim.x) {
      const int r = idx / K, c = idx % K;
      const int64_t m = c0 + r;
      sX[r * LDX + c] = m < r_end ? X[m * ldx + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int ks = 0; ks < kTile; ks += 16) {
      int q = 0;
      for (int tile = warp; tile < tiles; tile += 4, ++q) {
        const int mt = tile / nt_n, nt = tile % nt_n;
        const int rr = ks + 2 * t;
        const int c_lo = mt * 16 + g, c_hi = c_lo + 8;
        const uint32_t a0 = pack2(sY[rr * LDY + c_lo], sY[(rr + 1) * LDY + c_lo]);
        const uint32_t a1 = pack2(sY[rr * LDY + c_hi], sY[(rr + 1) * LDY + c_hi]);
        const uint32_t a2 = pack2(sY[(rr + 8) * LDY + c_lo], sY[(rr + 9) * LDY + c_lo]);
        const uint32_t a3 = pack2(sY[(rr + 8) * LDY + c_hi], sY[(rr + 9) * LDY + c_hi]);
        const int kc = nt * 8 + g;
        const uint32_t b0 = pack2(sX[rr * LDX + kc], sX[(rr + 1) * LDX + kc]);
        const uint32_t b1 = pack2(sX[(rr + 8) * LDX + kc], sX[(rr + 9) * LDX + kc]);
        mma16816(acc[q], a0, a1, a2, a3, b0, b1);
      }
    }
  }
  float* out = partial + (size_t)blockIdx.x * NO * K;
  int q = 0;
  for (int tile = warp; tile < tiles; tile += 4, ++q) {
    const int mt = tile / nt_n, nt = tile % nt_n;
    const int r0 = mt * 16 + g, col = nt * 8 + 2 * t;
    out[r0 * K + col] = acc[q][0];
    out[r0 * K + col + 1] = acc[q][1];
    out[(r0 + 8) * K + col] = acc[q][2];
    out[(r0 + 8) * K + col + 1] = acc[q][3];
  }
}

// grad[o] += sum over blocks b (in order) of partial[b][o]
__global__ void k_reduce_partials(int blocks, int count, const float* __restrict__ partial, float* __restrict__ grad) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= count) return;
  float s = 0.f;
  for (int b = 0; b < blocks; ++b) s += partial[(size_t)b * count + o];
  grad[o] += s;
}

// ------------------------------------------------------------------ graph and features
// Edge CSR of the frozen neighbour table: node i owns edges [off[i], off[i+1]), fluid
// neighbours first, then walls; nbr >= 0 is a fluid slot, nbr < 0 encodes wall -1 - w.
__global__ void k_edge_count(int64_t n, const uint32_t* __restrict__ nbc, uint32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = (nbc[i] & 0xffffu) + (nbc[i] >> 16);
}

// Node features (one 32-byte row per particle) and the edge list of the frozen table.
template <int D>
__global__ void k_node_features(int64_t n, const int4* __restrict__ P, const float4* __restrict__ V,
                                const int* __restrict__ inst_of, const Inst* __restrict__ inst,
                                const Ctrl* __restrict__ ctrl, const int* __restrict__ nbr,
                                const uint32_t* __restrict__ nbc, const uint32_t* __restrict__ off,
                                int* __restrict__ esrc, int* __restrict__ enbr, bf16* __restrict__ U) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = inst_of ? inst_of[i] : 0;
  const Inst& I = inst[k];
  const int4 pi = P[i];
  const float4 vi = V[i];
  const float inv_c0 = 1.0f / I.c0;
  const float uv[3] = {vi.x, vi.y, vi.z};
  __align__(16) bf16 u[16];
  for (int c = 0; c < 16; ++c) u[c] = __float2bfloat16_rn(0.f);
  for (int a = 0; a < D; ++a) u[a] = __float2bfloat16_rn(uv[a] * inv_c0);
  u[D] = __float2bfloat16_rn(S_RHO * (i2f(pi.w) / I.rho0));
  u[D + 1] = __float2bfloat16_rn((float)ctrl[k].dt_ad * I.c0 * I.inv_h);
  u[D + 2] = __float2bfloat16_rn(1.0f);
  uint4* dst = reinterpret_cast<uint4*>(U + i * 16);
  dst[0] = reinterpret_cast<const uint4*>(u)[0];
  dst[1] = reinterpret_cast<const uint4*>(u)[1];
  const uint32_t cnt = nbc[i];
  const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
  uint32_t e = off[i];
  for (int s = 0; s < nf + nw; ++s, ++e) {
    const bool wall = s >= nf;
    const int j = nbr[slot_index(n, i, wall ? wall_slot0(nf) + (s - nf) : s)];
    esrc[e] = (int)i;
    enbr[e] = wall ? -1 - j : j;
  }
}

// Static features of edge e, 16 bf16 per edge: [r_ij/h, (v_i - v_j)/c0, 100 dev_i,
// 100 dev_j, is_wall, 0...]; the rounds' input rows are assembled from them by k_edge_rows.
template <int D>
__global__ void k_edge_features(int64_t E, const int4* __restrict__ P, const float4* __restrict__ V,
                                const int* __restrict__ inst_of, const Inst* __restrict__ inst,
                                const int* __restrict__ esrc, const int* __restrict__ enbr,
                                const int4* __restrict__ WP, bf16* __restrict__ XS) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int i = esrc[e], jj = enbr[e];
  const bool wall = jj < 0;
  const int j = wall ? -1 - jj : jj;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const int4 pi = P[i];
  const float4 vi = V[i];
  const int4 pj = wall ? WP[j] : P[j];
  float4 vj = make_float4(0.f, 0.f, 0.f, 0.f);
  float dev_j = 0.f;
  if (!wall) {
    vj = V[j];
    dev_j = i2f(pj.w) / I.rho0;
  }
  const float inv_c0 = 1.0f / I.c0;
  const int qi[3] = {pi.x, pi.y, pi.z}, qj[3] = {pj.x, pj.y, pj.z};
  const float ui[3] = {vi.x, vi.y, vi.z}, uj[3] = {vj.x, vj.y, vj.z};
  __align__(16) bf16 row[16];
  for (int c = 0; c < 16; ++c) row[c] = __float2bfloat16_rn(0.f);
  for (int a = 0; a < D; ++a) {
    row[a] = __float2bfloat16_rn((float)wrap_diff(qi[a] - qj[a], I.period[a]) * I.dq * I.inv_h);
    row[D + a] = __float2bfloat16_rn((ui[a] - uj[a]) * inv_c0);
  }
  row[2 * D] = __float2bfloat16_rn(S_RHO * (i2f(pi.w) / I.rho0));
  row[2 * D + 1] = __float2bfloat16_rn(S_RHO * dev_j);
  row[2 * D + 2] = __float2bfloat16_rn(wall ? 1.0f : 0.0f);
  uint4* dst = reinterpret_cast<uint4*>(XS + e * 16);
  dst[0] = reinterpret_cast<const uint4*>(row)[0];
  dst[1] = reinterpret_cast<const uint4*>(row)[1];
}

// Round input row of edge e: XE[e] = [static features (fe) | bf16(h_j) (64, zero for a
// wall) | 1 | 0...] (80 columns). One thread per 16-byte piece: consecutive threads write
// consecutive pieces.
__global__ void k_edge_rows(int64_t E, int fe, const bf16* __restrict__ XS, const int* __restrict__ enbr,
                            const float* __restrict__ H, bf16* __restrict__ XE) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= E * 10) return;
  const int64_t e = idx / 10;
  const int c0 = (int)(idx - e * 10) * 8;
  const int j = enbr[e];
  __align__(16) bf16 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c = c0 + k;
    float x = 0.f;
    if (c < fe) x = __bfloat162float(XS[e * 16 + c]);
    else if (c < fe + F) x = j >= 0 ? H[(int64_t)j * F + (c - fe)] : 0.f;
    else if (c == fe + F) x = 1.0f;
    v[k] = __float2bfloat16_rn(x);
  }
  *reinterpret_cast<uint4*>(XE + e * 80 + c0) = *reinterpret_cast<const uint4*>(v);
}

// XN[i] = [bf16(h_i), bf16(a_i), 1], a_i = (1/nbar) sum over node i's edges of M
__global__ void k_segsum(int64_t n, const uint32_t* __restrict__ off, const float* __restrict__ Mm,
                         const float* __restrict__ H, float inv_nbar, bf16* __restrict__ XN) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  const int64_t i = idx / F;
  const int f = (int)(idx % F);
  float s = 0.f;
  for (uint32_t e = off[i]; e < off[i + 1]; ++e) s += Mm[(int64_t)e * F + f];
  XN[i * 144 + f] = __float2bfloat16_rn(H[i * F + f]);
  XN[i * 144 + F + f] = __float2bfloat16_rn(s * inv_nbar);
}

// Edge network of one round, fused for inference. Each warp takes a run of kFuseNodes
// nodes and walks their edges in 16-row tiles. The next tile's h_j rows and static edge
// features are loaded (whole rows, 16-byte pieces) while the current tile is multiplied,
// and the neighbour indices one tile ahead of that. A tile's A fragments are read from a
// per-warp staging copy of those rows, column by column as k_edge_rows lays a round input
// row out (static features, bf16(h_j) or zero for a wall, the bias 1, zero padding). Both
// edge layers run on the tensor cores (mma.sync m16n8k16, k-steps in k_dense's order; the
// first layer's accumulators become the second layer's A fragments after k_dense's ReLU
// and bfloat16 rounding), and the messages are added per node in edge order as k_segsum
// does. After its edges, the run's node rows go through the node network (both node
// layers, the update added to h) into the other node-state buffer. XN and the new node
// states are therefore bit-identical to the unfused path's, and no per-edge row,
// activation or message goes to memory.
constexpr int kFuseWarps = 8;
constexpr int kFuseNodes = 8;
constexpr int kFuseLd = 88;                   // padded weight row of 80 bf16
constexpr int kStageLd = 68;                  // staged h row: 64 floats + pad (16-byte rows)
constexpr int kStageWords = 16 * kStageLd + 16 * 8;   // h rows, then the static features (bf16 pairs)
constexpr int kMsgLd = 72;                    // message row stride: conflict-free float2 stores

static_assert(16 * kMsgLd <= kStageWords, "messages must fit the staging area");

constexpr int kNodeLd = 152;                  // padded weight row of 144 bf16 (node layer 1)

inline size_t fused_smem() {
  return (size_t)(3 * 64 * kFuseLd + 64 * kNodeLd) * sizeof(bf16) + (size_t)kFuseWarps * kStageWords * sizeof(float);
}

// column of slot q (0..19) of a lane with quad index t: k-step q / 4, position q % 4 in
// {0, 1, 8, 9}
__device__ __forceinline__ int fuse_col(int q, int t) { return (q >> 2) * 16 + 2 * t + (q & 1) + ((q >> 1) & 1) * 8; }

// B fragments of two n-tiles (nt, nt + 1) at k-step k0 from a row-major [n][kFuseLd] weight
// copy: lane i addresses row i % 8 of 8x8 matrix i / 8 (matrices: (nt, k0), (nt, k0 + 8),
// (nt + 1, k0), (nt + 1, k0 + 8)), and receives row lane / 4, columns 2 (lane % 4), +1 of
// each, which is the m16n8k16 B fragment.
template <int LD = kFuseLd>
__device__ __forceinline__ void ldsm_b4(const bf16* W, int nt, int k0, int lane, uint32_t& b0, uint32_t& b1,
                                        uint32_t& c0, uint32_t& c1) {
  const int m = lane >> 3;
  const bf16* p = W + ((nt + (m >> 1)) * 8 + (lane & 7)) * LD + k0 + (m & 1) * 8;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(b0), "=r"(b1), "=r"(c0), "=r"(c1)
               : "r"(a));
}

// bf16 of column c of a staged row: static feature, h value, bias or zero padding
template <int FE>
__device__ __forceinline__ bf16 fuse_elem(const float* __restrict__ hrow, const bf16* __restrict__ xrow, int c,
                                          bool valid) {
  if (c < FE) return xrow[c];
  if (c < FE + F) return __float2bfloat16_rn(hrow[c - FE]);
  return __float2bfloat16_rn(valid && c == FE + F ? 1.0f : 0.f);
}

template <int FE>
__global__ void __launch_bounds__(kFuseWarps * 32, 2)
k_edge_round_fused(int64_t n, const uint32_t* __restrict__ off, const bf16* __restrict__ XS,
                   const int* __restrict__ enbr, const float* __restrict__ H, const bf16* __restrict__ W1,
                   const bf16* __restrict__ W2, const bf16* __restrict__ Wn1, const bf16* __restrict__ Wn2,
                   float inv_nbar, bf16* __restrict__ XN, float* __restrict__ Hout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  bf16* sW1 = reinterpret_cast<bf16*>(smem_raw);
  bf16* sW2 = sW1 + 64 * kFuseLd;
  bf16* sN2 = sW2 + 64 * kFuseLd;             // node layer 2, rows of kFuseLd
  bf16* sN1 = sN2 + 64 * kFuseLd;             // node layer 1, rows of kNodeLd
  float* stage = reinterpret_cast<float*>(sN1 + 64 * kNodeLd) + warp * kStageWords;   // h rows
  bf16* xstage = reinterpret_cast<bf16*>(stage + 16 * kStageLd);                       // [16][16]
  float* sM = stage;                          // the messages reuse the staging rows (16 x kMsgLd)
  for (int idx = threadIdx.x; idx < 64 * 10; idx += blockDim.x) {
    const int r = idx / 10, c = (idx % 10) * 8;
    *reinterpret_cast<uint4*>(&sW1[r * kFuseLd + c]) = *reinterpret_cast<const uint4*>(&W1[r * 80 + c]);
    *reinterpret_cast<uint4*>(&sW2[r * kFuseLd + c]) = *reinterpret_cast<const uint4*>(&W2[r * 80 + c]);
    *reinterpret_cast<uint4*>(&sN2[r * kFuseLd + c]) = *reinterpret_cast<const uint4*>(&Wn2[r * 80 + c]);
  }
  for (int idx = threadIdx.x; idx < 64 * 18; idx += blockDim.x) {
    const int r = idx / 18, c = (idx % 18) * 8;
    *reinterpret_cast<uint4*>(&sN1[r * kNodeLd + c]) = *reinterpret_cast<const uint4*>(&Wn1[r * 144 + c]);
  }
  __syncthreads();
  const int64_t chunks = (n + kFuseNodes - 1) / kFuseNodes;
  for (int64_t ch = (int64_t)blockIdx.x * kFuseWarps + warp; ch < chunks; ch += (int64_t)gridDim.x * kFuseWarps) {
    const int64_t i0 = ch * kFuseNodes, i1 = min(i0 + (int64_t)kFuseNodes, n);
    const uint32_t e_begin = off[i0], e_end = off[i1];
    int64_t cur = i0;                         // node whose sum is open
    uint32_t cur_end = off[cur + 1];
    float s0 = 0.f, s1 = 0.f;                 // this lane's columns 2 lane, 2 lane + 1
    // close every node whose edges end at or before edge e (edgeless nodes included)
    auto close_until = [&](uint32_t e) {
      while (cur < i1 && cur_end <= e) {
        const int f = 2 * lane;
        const float2 hv = *reinterpret_cast<const float2*>(&H[cur * F + f]);
        *reinterpret_cast<uint32_t*>(&XN[cur * 144 + f]) = pack2(__float2bfloat16_rn(hv.x), __float2bfloat16_rn(hv.y));
        *reinterpret_cast<uint32_t*>(&XN[cur * 144 + F + f]) =
            pack2(__float2bfloat16_rn(s0 * inv_nbar), __float2bfloat16_rn(s1 * inv_nbar));
        s0 = s1 = 0.f;
        ++cur;
        if (cur < i1) cur_end = off[cur + 1];
      }
    };
    close_until(e_begin);
    // neighbour index of row `lane` (lanes 0..15) of the tile at t0, -1 past the end
    auto idx_of = [&](uint32_t t0) { return lane < 16 && t0 + lane < e_end ? __ldg(&enbr[t0 + lane]) : -1; };
    // the tile's rows: piece p of lane l is row 2p + l / 16, floats 4 (l % 16) .. + 3
    float4 hq[8];
    uint4 xq;
    auto load_tile = [&](uint32_t t0, int jrow) {
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const int row = 2 * p + (lane >> 4);
        const int j = __shfl_sync(0xffffffffu, jrow, row);
        hq[p] = (t0 + row < e_end && j >= 0) ? __ldg(reinterpret_cast<const float4*>(&H[(int64_t)j * F]) + (lane & 15))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const int xrow = lane >> 1;
      xq = t0 + xrow < e_end ? __ldg(reinterpret_cast<const uint4*>(&XS[((int64_t)t0 + xrow) * 16]) + (lane & 1))
                             : make_uint4(0u, 0u, 0u, 0u);
    };
    load_tile(e_begin, idx_of(e_begin));
    int jn = idx_of(e_begin + 16);
    for (uint32_t t0 = e_begin; t0 < e_end; t0 += 16) {
      // stage the current tile's rows and read this lane's A fragments of the first layer
#pragma unroll
      for (int p = 0; p < 8; ++p)
        *reinterpret_cast<float4*>(&stage[(2 * p + (lane >> 4)) * kStageLd + 4 * (lane & 15)]) = hq[p];
      *reinterpret_cast<uint4*>(&xstage[(lane >> 1) * 16 + 8 * (lane & 1)]) = xq;
      __syncwarp();
      const bool va = t0 + g < e_end, vb = t0 + g + 8 < e_end;
      const float* ha = stage + g * kStageLd;
      const float* hb = ha + 8 * kStageLd;
      const bf16* xa = xstage + g * 16;
      const bf16* xb = xa + 8 * 16;
      uint32_t A[5][4];
#pragma unroll
      for (int kk = 0; kk < 5; ++kk) {
        const int c = kk * 16 + 2 * t;
        A[kk][0] = pack2(fuse_elem<FE>(ha, xa, c, va), fuse_elem<FE>(ha, xa, c + 1, va));
        A[kk][1] = pack2(fuse_elem<FE>(hb, xb, c, vb), fuse_elem<FE>(hb, xb, c + 1, vb));
        A[kk][2] = pack2(fuse_elem<FE>(ha, xa, c + 8, va), fuse_elem<FE>(ha, xa, c + 9, va));
        A[kk][3] = pack2(fuse_elem<FE>(hb, xb, c + 8, vb), fuse_elem<FE>(hb, xb, c + 9, vb));
      }
      __syncwarp();                           // staging read: free for the messages
      // next tile's rows in flight during this tile's products
      const uint32_t t1 = t0 + 16;
      if (t1 < e_end) {
        load_tile(t1, jn);
        jn = idx_of(t1 + 16);
      }
      float acc[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 5; ++kk)
#pragma unroll
        for (int nt = 0; nt < 8; nt += 2) {
          uint32_t b0, b1, c0, c1;
          ldsm_b4(sW1, nt, kk * 16, lane, b0, b1, c0, c1);
          mma16816(acc[nt], A[kk][0], A[kk][1], A[kk][2], A[kk][3], b0, b1);
          mma16816(acc[nt + 1], A[kk][0], A[kk][1], A[kk][2], A[kk][3], c0, c1);
        }
      // second layer: A = [bf16(relu(z)) | 1 | 0...], z's fragments reused in place
      float acc2[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) acc2[nt][0] = acc2[nt][1] = acc2[nt][2] = acc2[nt][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 5; ++kk) {
        uint32_t a0, a1, a2, a3;
        if (kk < 4) {
          const float* lo = acc[2 * kk];
          const float* hi = acc[2 * kk + 1];
          a0 = pack2(__float2bfloat16_rn(fmaxf(lo[0], 0.f)), __float2bfloat16_rn(fmaxf(lo[1], 0.f)));
          a1 = pack2(__float2bfloat16_rn(fmaxf(lo[2], 0.f)), __float2bfloat16_rn(fmaxf(lo[3], 0.f)));
          a2 = pack2(__float2bfloat16_rn(fmaxf(hi[0], 0.f)), __float2bfloat16_rn(fmaxf(hi[1], 0.f)));
          a3 = pack2(__float2bfloat16_rn(fmaxf(hi[2], 0.f)), __float2bfloat16_rn(fmaxf(hi[3], 0.f)));
        } else {                              // columns 64..79: the bias column, then zeros
          a0 = a1 = t == 0 ? pack2(__float2bfloat16_rn(1.0f), __float2bfloat16_rn(0.f)) : 0u;
          a2 = a3 = 0u;
        }
#pragma unroll
        for (int nt = 0; nt < 8; nt += 2) {
          uint32_t b0, b1, c0, c1;
          ldsm_b4(sW2, nt, kk * 16, lane, b0, b1, c0, c1);
          mma16816(acc2[nt], a0, a1, a2, a3, b0, b1);
          mma16816(acc2[nt + 1], a0, a1, a2, a3, c0, c1);
        }
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = nt * 8 + 2 * t;
        *reinterpret_cast<float2*>(&sM[g * kMsgLd + c]) = make_float2(acc2[nt][0], acc2[nt][1]);
        *reinterpret_cast<float2*>(&sM[(g + 8) * kMsgLd + c]) = make_float2(acc2[nt][2], acc2[nt][3]);
      }
      __syncwarp();
      const int rows = (int)min(16u, e_end - t0);
      for (int r = 0; r < rows; ++r) {
        close_until(t0 + (uint32_t)r);
        const float2 m = *reinterpret_cast<const float2*>(&sM[r * kMsgLd + 2 * lane]);
        s0 += m.x;
        s1 += m.y;
      }
      __syncwarp();                           // sM free for the next tile's staging
    }
    close_until(e_end);
    // node network of the run's nodes (the rows of one MMA tile), as the unfused node layers
    // compute it: z = relu(W_n1 XN), h_out = h + W_n2 [z, 1]
    __syncwarp();                             // the run's XN rows, written above, visible
    const int nrows = (int)(i1 - i0);
    const bool vg = g < nrows, vh = g + 8 < nrows;
    const bf16* xn = XN + (i0 + g) * 144;
    const bf16* xh = xn + 8 * 144;
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 9; ++kk) {
      const uint32_t a0 = vg ? ld_u32(xn + kk * 16 + 2 * t) : 0u;
      const uint32_t a1 = vh ? ld_u32(xh + kk * 16 + 2 * t) : 0u;
      const uint32_t a2 = vg ? ld_u32(xn + kk * 16 + 2 * t + 8) : 0u;
      const uint32_t a3 = vh ? ld_u32(xh + kk * 16 + 2 * t + 8) : 0u;
#pragma unroll
      for (int nt = 0; nt < 8; nt += 2) {
        uint32_t b0, b1, c0, c1;
        ldsm_b4<kNodeLd>(sN1, nt, kk * 16, lane, b0, b1, c0, c1);
        mma16816(acc[nt], a0, a1, a2, a3, b0, b1);
        mma16816(acc[nt + 1], a0, a1, a2, a3, c0, c1);
      }
    }
    float acc2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc2[nt][0] = acc2[nt][1] = acc2[nt][2] = acc2[nt][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 5; ++kk) {
      uint32_t a0, a1, a2, a3;
      if (kk < 4) {
        const float* lo = acc[2 * kk];
        const float* hi = acc[2 * kk + 1];
        a0 = pack2(__float2bfloat16_rn(fmaxf(lo[0], 0.f)), __float2bfloat16_rn(fmaxf(lo[1], 0.f)));
        a1 = pack2(__float2bfloat16_rn(fmaxf(lo[2], 0.f)), __float2bfloat16_rn(fmaxf(lo[3], 0.f)));
        a2 = pack2(__float2bfloat16_rn(fmaxf(hi[0], 0.f)), __float2bfloat16_rn(fmaxf(hi[1], 0.f)));
        a3 = pack2(__float2bfloat16_rn(fmaxf(hi[2], 0.f)), __float2bfloat16_rn(fmaxf(hi[3], 0.f)));
      } else {
        a0 = a1 = t == 0 ? pack2(__float2bfloat16_rn(1.0f), __float2bfloat16_rn(0.f)) : 0u;
        a2 = a3 = 0u;
      }
#pragma unroll
      for (int nt = 0; nt < 8; nt += 2) {
        uint32_t b0, b1, c0, c1;
        ldsm_b4(sN2, nt, kk * 16, lane, b0, b1, c0, c1);
        mma16816(acc2[nt], a0, a1, a2, a3, b0, b1);
        mma16816(acc2[nt + 1], a0, a1, a2, a3, c0, c1);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int64_t o = (i0 + g) * F + nt * 8 + 2 * t;
      if (vg) {
        const float2 h = *reinterpret_cast<const float2*>(&H[o]);
        *reinterpret_cast<float2*>(&Hout[o]) = make_float2(h.x + acc2[nt][0], h.y + acc2[nt][1]);
      }
      if (vh) {
        const float2 h = *reinterpret_cast<const float2*>(&H[o + 8 * F]);
        *reinterpret_cast<float2*>(&Hout[o + 8 * F]) = make_float2(h.x + acc2[nt][2], h.y + acc2[nt][3]);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ fused edge round, pipelined (tcgen05)
// Round input row templates: T[j] is edge row [XS | bf16(h_j) | 1 | 0...] of any edge whose
// neighbour is fluid node j, with zeros where the static features go; T[n] serves wall
// neighbours (h = 0). An edge row is its neighbour's template with the static features
// merged into the first one or two 16-byte pieces. The same launch writes the h part of
// the round's node rows, XN[i][0, 64) = bf16(h_i). One thread per 16-byte piece.
template <int FE>
__global__ void k_node_templates(int64_t n, const float* __restrict__ H, bf16* __restrict__ T,
                                 bf16* __restrict__ XN) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  __align__(16) bf16 v[8];
  if (idx < (n + 1) * 10) {
    const int64_t j = idx / 10;
    const int c0 = (int)(idx - j * 10) * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = c0 + k;
      float x = 0.f;
      if (c >= FE && c < FE + F) x = j < n ? H[j * F + (c - FE)] : 0.f;
      else if (c == FE + F) x = 1.0f;
      v[k] = __float2bfloat16_rn(x);
    }
    *reinterpret_cast<uint4*>(T + j * 80 + c0) = *reinterpret_cast<const uint4*>(v);
  } else if (idx < (n + 1) * 10 + n * 8) {
    const int64_t q = idx - (n + 1) * 10, i = q / 8;
    const int c0 = (int)(q - i * 8) * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __float2bfloat16_rn(H[i * F + c0 + k]);
    *reinterpret_cast<uint4*>(XN + i * 144 + c0) = *reinterpret_cast<const uint4*>(v);
  }
}

// Edge network of one round for inference on the fifth-generation tensor cores, as a
// warp-specialised pipeline. Each CTA takes runs of at most kWsRun consecutive nodes and
// walks their edges in 128-row tiles through a ring of kWsStages tile buffers:
//   warp 4 + p (producer p) assembles the tiles t with t % kWsStages == p in buffer p:
//     pieces of the neighbours' templates by cp.async, the static features merged into
//     the first pieces by plain stores; it signals a tile as soon as its copies have landed;
//   warp 4 + kWsStages (one issuing lane) runs layer 1 of tile t + 1 into TMEM accumulator set
//     (t + 1) % 2 before layer 2 of tile t, each as K/16 tcgen05.mma (M = 128, N = 64)
//     committed to an mbarrier; layer 2's commit also frees the tile buffer;
//   warps 0-3 (epilogue, one TMEM lane = one edge row per thread) turn layer 1's
//     accumulators of tile t into bf16(relu(z)) and the constant columns, written over the
//     tile's own buffer as layer 2's A operand; then, while layer 2 of tile t runs, they
//     stage the messages of tile t - 1 32 columns at a time and add them per node in edge
//     order (a node whose edges continue into the next tile carries its partial sums);
//     closed nodes write XN[i][64, 128) = bf16(a_i).
// Every product, rounding and sum is the layer-by-layer path's, so XN is bit-identical to
// it; the node layers then run as that path's dense layers. Every wait is bounded: one that
// runs out sets ERR_TIMEOUT in *err and makes every role stop. On GB300 this pipeline runs
// the 100,128-particle learned step in 1.17 ms against 1.15 ms for the warp-level MMA rounds
// (k_edge_round_fused): the epilogue warpgroup's per-node sums and operand conversion,
// not the tensor core, bound it, so inference keeps the warp-level rounds by default.
constexpr int kWsStages = 3;
constexpr int kWsThreads = 128 + 32 * kWsStages + 32;   // warps 0-3 epilogue, one producer per buffer, MMA
constexpr int kWsMmaWarp = 4 + kWsStages;
constexpr int kWsRun = 128;                   // nodes in a run, at most
constexpr int kWsTile = 128 * 80 * 2;         // bytes of one 128-row tile of edge rows
constexpr int kWsMsgLd = 36;                  // staged message row: 32 floats + pad (16-byte rows, conflict-free)

inline size_t ws_smem() {
  // at least a third of an SM's shared memory, so that no more than two CTAs (256 TMEM
  // columns each) share an SM and a TMEM allocation never waits
  const size_t need = (size_t)2 * 64 * 80 * 2 + (size_t)kWsStages * kWsTile + 128 * kWsMsgLd * sizeof(float) +
                      2 * 64 * sizeof(float) + (kWsRun + 1) * sizeof(uint32_t);
  return std::max(need, (size_t)233472 / 3 + 1);
}

struct WsSync {
  uint64_t full[kWsStages], empty[kWsStages];   // tile buffer written / free again
  uint64_t a1_full[2], a1_empty[2];             // layer-1 accumulators ready / read
  uint64_t a2_ready[2];                         // layer 2's operand written
  uint64_t a2_full[2], a2_empty[2];             // layer-2 accumulators ready / read
  uint64_t fin;                                 // every MMA of the CTA complete
  int abort;
};

__device__ __forceinline__ void ws_bar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tc::smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void ws_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void ws_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(tc::smem_u32(bar))
               : "memory");
}
// Bounded wait for the phase of parity `parity`; gives up when another role has aborted,
// and aborts every role when it runs out itself.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* err) {
  for (unsigned spin = 0; spin < tc::kWaitLimit; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(tc::smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort) return false;
  }
  *abort = 1;
  atomicOr(err, ERR_TIMEOUT);
  return false;
}
// AND of a flag over the epilogue warpgroup (named barrier 1, 128 threads): the same
// decision in every epilogue thread
__device__ __forceinline__ bool epi_all(bool v) {
  int r;
  asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\tbar.red.and.pred q, 1, 128, p;\n\t"
               "selp.s32 %0, 1, 0, q;\n\t}\n"
               : "=r"(r)
               : "r"((int)v)
               : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }
__device__ __forceinline__ float ld_shared_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
// number of epilogue threads whose flag is set (named barrier 1, 128 threads)
__device__ __forceinline__ int epi_count(bool v) {
  int r;
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %1, 0;\n\tbar.red.popc.u32 %0, 1, 128, p;\n\t}\n"
               : "=r"(r)
               : "r"((int)v)
               : "memory");
  return r;
}

template <int FE>
__global__ void __launch_bounds__(kWsThreads, 2)
k_edge_round_ws(int64_t n, int run, const uint32_t* __restrict__ off, const bf16* __restrict__ XS,
                const int* __restrict__ enbr, const bf16* __restrict__ T, const bf16* __restrict__ W1,
                const bf16* __restrict__ W2, float inv_nbar, bf16* __restrict__ XN, int* __restrict__ err) {
  constexpr int MP = (FE + 7) / 8;                    // leading pieces that hold static features
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ WsSync S;
  __shared__ uint32_t tmem_slot;
  __shared__ int carry_open;
  unsigned char* sW1 = tc_smem;                       // 64 x 80
  unsigned char* sW2 = sW1 + 64 * 80 * 2;             // 64 x 80
  unsigned char* sTiles = sW2 + 64 * 80 * 2;          // kWsStages x (128 x 80)
  float* stage = reinterpret_cast<float*>(sTiles + kWsStages * kWsTile);   // 128 x 32 messages
  float* carry_in = stage + 128 * kWsMsgLd;           // partial sums of the node carried into the tile
  float* carry_out = carry_in + 64;                   // ... and of the node it leaves open
  uint32_t* soff = reinterpret_cast<uint32_t*>(carry_out + 64);   // the run's edge offsets
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  load_operand<false>(sW1, 64, 80, W1, 80, 64);
  load_operand<false>(sW2, 64, 80, W2, 80, 64);
  if (tid == 0) {
    for (int s = 0; s < kWsStages; ++s) {
      ws_bar_init(&S.full[s], 1);
      ws_bar_init(&S.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ws_bar_init(&S.a1_full[b], 1);
      ws_bar_init(&S.a1_empty[b], 4);             // one arrival per epilogue warp
      ws_bar_init(&S.a2_ready[b], 4);
      ws_bar_init(&S.a2_full[b], 1);
      ws_bar_init(&S.a2_empty[b], 4);
    }
    ws_bar_init(&S.fin, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, 256);
  tc::fence_to_async();                               // the weights, for the tensor core
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;                    // acc1[b] at 64 b, acc2[b] at 128 + 64 b
  volatile int* abort = &S.abort;
  const int64_t runs = (n + run - 1) / run;

  if (warp >= 4 && warp < kWsMmaWarp) {
    // ---------------- producers: warp 4 + p assembles the tiles t with t % kWsStages == p,
    // always into buffer p, and signals each as soon as its copies have landed
    const int p = warp - 4;
    uint32_t t = 0;
    bool ok = true;
    for (int64_t rr = blockIdx.x; rr < runs && ok; rr += gridDim.x) {
      const int64_t i0 = rr * run, i1 = min(i0 + (int64_t)run, n);
      const uint32_t E0 = __ldg(&off[i0]), E1 = __ldg(&off[i1]);
      for (uint32_t e0 = E0; e0 < E1; e0 += 128, ++t) {
        if ((int)(t % kWsStages) != p) continue;
        const bool got = ws_wait(&S.empty[p], ((t / kWsStages) & 1u) ^ 1u, abort, err);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        const uint32_t te = min(e0 + 128u, E1);
        unsigned char* A = sTiles + p * kWsTile;
        // rows lane + 32 k: every load of the tile issued before any is used
        int jr[4];
        bool vr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t e = e0 + (uint32_t)(lane + 32 * k);
          vr[k] = e < te;
          const int j = vr[k] ? __ldg(&enbr[e]) : 0;
          jr[k] = j < 0 ? (int)n : j;                 // walls: the zero template
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bf16* tj = T + (int64_t)jr[k] * 80;
#pragma unroll
          for (int q = MP; q < 10; ++q)
            cp_async16(A + tc::core_offset(128, lane + 32 * k, q * 8), vr[k] ? tj + q * 8 : T, vr[k]);
        }
        uint4 q[4][MP], x[4][MP];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int c = 0; c < MP; ++c) {
            q[k][c] = x[k][c] = make_uint4(0u, 0u, 0u, 0u);
            if (vr[k]) {
              q[k][c] = __ldg(reinterpret_cast<const uint4*>(T + (int64_t)jr[k] * 80) + c);
              x[k][c] = __ldg(reinterpret_cast<const uint4*>(XS + (int64_t)(e0 + lane + 32 * k) * 16) + c);
            }
          }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int c = 0; c < MP; ++c) {
            bf16* a = reinterpret_cast<bf16*>(&q[k][c]);
            const bf16* xa = reinterpret_cast<const bf16*>(&x[k][c]);
#pragma unroll
            for (int m = 0; m < 8; ++m)
              if (c * 8 + m < FE) a[m] = xa[m];
            *reinterpret_cast<uint4*>(A + tc::core_offset(128, lane + 32 * k, c * 8)) = q[k][c];
          }
        cp_async_commit();
        cp_async_wait_all();
        tc::fence_to_async();
        __syncwarp();                                 // the warp's copies and stores, then one arrival
        if (lane == 0) ws_arrive(&S.full[p]);
      }
    }
    cp_async_wait_all();
  } else if (warp == kWsMmaWarp) {
    // ---------------- MMA issue (all lanes wait, lane 0 issues)
    uint32_t TT = 0;
    for (int64_t rr = blockIdx.x; rr < runs; rr += gridDim.x) {
      const int64_t i0 = rr * run, i1 = min(i0 + (int64_t)run, n);
      const uint32_t E0 = __ldg(&off[i0]), E1 = __ldg(&off[i1]);
      TT += (E1 - E0 + 127u) / 128u;
    }
    const uint32_t w1 = tc::smem_u32(sW1), w2 = tc::smem_u32(sW2);
    auto layer1 = [&](uint32_t t) -> bool {
      const int s = (int)(t % kWsStages), b = (int)(t & 1u);
      bool g = ws_wait(&S.full[s], (t / kWsStages) & 1u, abort, err);
      g = g && ws_wait(&S.a1_empty[b], ((t >> 1) & 1u) ^ 1u, abort, err);
      if (!__all_sync(0xffffffffu, g)) return false;
      tc::fence_after_sync();
      if (lane == 0) tc::mma_tile<64>(tmem + 64 * b, tc::smem_u32(sTiles + s * kWsTile), w1, 80, false, &S.a1_full[b]);
      __syncwarp();
      return true;
    };
    bool ok = TT == 0 || layer1(0);
    for (uint32_t t = 0; t < TT && ok; ++t) {
      if (t + 1 < TT && !layer1(t + 1)) break;
      const int s = (int)(t % kWsStages), b = (int)(t & 1u);
      bool g = ws_wait(&S.a2_ready[b], (t >> 1) & 1u, abort, err);
      g = g && ws_wait(&S.a2_empty[b], ((t >> 1) & 1u) ^ 1u, abort, err);
      if (!__all_sync(0xffffffffu, g)) break;
      tc::fence_after_sync();
      if (lane == 0) {
        tc::mma_tile<64>(tmem + 128 + 64 * b, tc::smem_u32(sTiles + s * kWsTile), w2, 80, false, &S.a2_full[b]);
        ws_commit(&S.empty[s]);                       // the tile buffer is free once layer 2 has read it
      }
      __syncwarp();
    }
    if (lane == 0) ws_commit(&S.fin);                 // every MMA issued above, complete
    __syncwarp();
    if (!tc::mbar_wait(&S.fin, 0) && lane == 0) atomicOr(err, ERR_TIMEOUT);
  } else {
    // ---------------- epilogue (warps 0-3): the messages of tile t - 1 are summed while
    // layer 2 of tile t runs (within a run; its last tile is summed before the next run)
    __align__(16) bf16 one[8];                        // layer 2's constant columns: 1 at 64, 0 after
#pragma unroll
    for (int k = 0; k < 8; ++k) one[k] = __float2bfloat16_rn(k == 0 ? 1.0f : 0.0f);
    uint32_t t = 0;
    bool ok = true;
    int cur = 0;                                      // first node of the run not yet closed
    int64_t i0 = 0;
    int nodes = 0;
    // messages of tile u = [e0, te) of the current run, summed per node in edge order. The
    // tile's nodes are cur, cur + 1, ... while their first edge lies before te (soff never
    // decreases, so they are the nodes cur + k with soff[cur + k] < te; an edgeless node
    // closes where it sits in edge order, those after the run's last edge close after its
    // last tile); a node whose edges run past te stays open and carries its sums.
    auto messages = [&](uint32_t u, uint32_t e0, uint32_t te) -> bool {
      const int b = (int)(u & 1u);
      const int k = cur + tid;
      const int len = epi_count(k < nodes && soff[k] < te);
      if (!epi_all(ws_wait(&S.a2_full[b], (u >> 1) & 1u, abort, err))) return false;
      tc::fence_after_sync();
#pragma unroll 1
      for (int c0 = 0; c0 < 64; c0 += 32) {
        float m[16];
        tc::tmem_ld16(tc::tmem_addr(tmem + 128 + 64 * b, warp, c0), m);
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4*>(&stage[tid * kWsMsgLd + q]) = make_float4(m[q], m[q + 1], m[q + 2], m[q + 3]);
        tc::tmem_ld16(tc::tmem_addr(tmem + 128 + 64 * b, warp, c0 + 16), m);
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4*>(&stage[tid * kWsMsgLd + 16 + q]) = make_float4(m[q], m[q + 1], m[q + 2], m[q + 3]);
        epi_sync();
        // two (node, column) sums a thread at a time, each over its rows in edge order, eight
        // rows' loads in flight (+0 past a node's last row leaves a sum that started at +0
        // unchanged, bit for bit)
        for (int p0 = tid; p0 < len * 32; p0 += 256) {
          const int p1 = p0 + 128;
          const bool two = p1 < len * 32;
          const int li0 = p0 >> 5, li1 = two ? p1 >> 5 : li0, q = p0 & 31;
          const uint32_t kb0 = soff[cur + li0], ke0 = soff[cur + li0 + 1];
          const uint32_t kb1 = soff[cur + li1], ke1 = soff[cur + li1 + 1];
          const int rb0 = (int)(max(kb0, e0) - e0), re0 = (int)(min(ke0, te) - e0);
          const int rb1 = (int)(max(kb1, e0) - e0), re1 = two ? (int)(min(ke1, te) - e0) : rb1;
          float s0 = (li0 == 0 && carry_open) ? carry_in[c0 + q] : 0.f;
          float s1 = (li1 == 0 && carry_open) ? carry_in[c0 + q] : 0.f;
          const uint32_t col = tc::smem_u32(stage + q);
          for (int r = 0; r < re0 - rb0 || r < re1 - rb1; r += 8) {
            float v[8], w[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              v[c] = ld_shared_f32(col + 4u * (uint32_t)(min(rb0 + r + c, 127) * kWsMsgLd));
              w[c] = ld_shared_f32(col + 4u * (uint32_t)(min(rb1 + r + c, 127) * kWsMsgLd));
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              s0 += rb0 + r + c < re0 ? v[c] : 0.f;
              s1 += rb1 + r + c < re1 ? w[c] : 0.f;
            }
          }
          if (ke0 <= te) XN[(i0 + cur + li0) * 144 + F + c0 + q] = __float2bfloat16_rn(s0 * inv_nbar);
          else carry_out[c0 + q] = s0;
          if (two) {
            if (ke1 <= te) XN[(i0 + cur + li1) * 144 + F + c0 + q] = __float2bfloat16_rn(s1 * inv_nbar);
            else carry_out[c0 + q] = s1;
          }
        }
        epi_sync();
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) ws_arrive(&S.a2_empty[b]);
      const bool open = len > 0 && soff[cur + len] > te;   // the tile's last node continues
      if (tid < 64) carry_in[tid] = carry_out[tid];   // read only after the barrier below
      if (tid == 0) carry_open = open ? 1 : 0;
      cur += open ? len - 1 : len;
      epi_sync();
      return true;
    };
    for (int64_t rr = blockIdx.x; rr < runs && ok; rr += gridDim.x) {
      i0 = rr * run;
      const int64_t i1 = min(i0 + (int64_t)run, n);
      nodes = (int)(i1 - i0);
      for (int k = tid; k <= nodes; k += 128) soff[k] = off[i0 + k];
      if (tid == 0) carry_open = 0;
      epi_sync();
      const uint32_t E0 = soff[0], E1 = soff[nodes];
      cur = 0;
      bool pending = false;                           // a tile whose messages are not summed yet
      uint32_t pu = 0, pe0 = 0, pte = 0;
      for (uint32_t e0 = E0; e0 < E1; e0 += 128, ++t) {
        const uint32_t te = min(e0 + 128u, E1);
        const int s = (int)(t % kWsStages), b = (int)(t & 1u);
        unsigned char* A = sTiles + s * kWsTile;
        // layer 2's A over the tile's rows: bf16(relu(z)) of this thread's row, 1, 0...
        if (!epi_all(ws_wait(&S.a1_full[b], (t >> 1) & 1u, abort, err))) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 16) {
          float z[16];
          tc::tmem_ld16(tc::tmem_addr(tmem + 64 * b, warp, c0), z);
          __align__(16) __nv_bfloat162 v[8];         // pairs rounded by one packed conversion each
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = __floats2bfloat162_rn(fmaxf(z[2 * q], 0.f), fmaxf(z[2 * q + 1], 0.f));
          *reinterpret_cast<uint4*>(A + tc::core_offset(128, tid, c0)) = *reinterpret_cast<const uint4*>(v);
          *reinterpret_cast<uint4*>(A + tc::core_offset(128, tid, c0 + 8)) = *reinterpret_cast<const uint4*>(v + 4);
        }
        *reinterpret_cast<uint4*>(A + tc::core_offset(128, tid, 64)) = *reinterpret_cast<const uint4*>(one);
        *reinterpret_cast<uint4*>(A + tc::core_offset(128, tid, 72)) = make_uint4(0u, 0u, 0u, 0u);
        tc::fence_to_async();
        tc::fence_before_sync();
        __syncwarp();                                 // the warp's TMEM reads and stores, then one arrival
        if (lane == 0) {
          ws_arrive(&S.a1_empty[b]);
          ws_arrive(&S.a2_ready[b]);
        }
        if (pending && !messages(pu, pe0, pte)) {
          ok = false;
          break;
        }
        pending = true;
        pu = t;
        pe0 = e0;
        pte = te;
      }
      if (ok && pending && !messages(pu, pe0, pte)) ok = false;
      if (!ok) break;
      // nodes left (edgeless ones after the run's last edge): a = 0
      for (int k = cur + tid / 64; k < nodes; k += 2)
        XN[(i0 + k) * 144 + F + (tid & 63)] = __float2bfloat16_rn(0.f * inv_nbar);
      epi_sync();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, 256);
  }
}

__global__ void k_rows_bf16(int64_t n, int cols, const float* __restrict__ src, int lds, bf16* __restrict__ dst,
                            int ldd) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * cols) return;
  const int64_t r = idx / cols;
  const int c = (int)(idx % cols);
  dst[r * ldd + c] = __float2bfloat16_rn(src[r * lds + c]);
}

// constant columns of an activation buffer: column `one` = 1, [pad_from, ld) = 0
__global__ void k_const_cols(int64_t rows, int ld, int one, int pad_from, bf16* __restrict__ A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  A[r * ld + one] = __float2bfloat16_rn(1.0f);
  for (int c = pad_from; c < ld; ++c) A[r * ld + c] = __float2bfloat16_rn(0.f);
}

// loss and its gradient: dY = 2 (y - target) / (n (d+1)) on the first d+1 columns
__global__ void k_loss(int64_t n, int dout, const float* __restrict__ Y, const double* __restrict__ T,
                       const int* __restrict__ id, bf16* __restrict__ dY, double* __restrict__ loss) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    const int64_t row = id[i];
    const double scale = 2.0 / ((double)n * dout);
    for (int c = 0; c < 16; ++c) {
      float gval = 0.f;
      if (c < dout) {
        const double d = (double)Y[i * 16 + c] - T[row * dout + c];
        l += d * d;
        gval = (float)(scale * d);
      }
      dY[i * 16 + c] = __float2bfloat16_rn(gval);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / ((double)n * dout));
}

// dh += dXN[:, :F]; dM[e] = bf16(dXN[src(e), F + f] / nbar)
__global__ void k_node_back(int64_t n, const float* __restrict__ dXN, float* __restrict__ dH) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  const int64_t i = idx / F;
  const int f = (int)(idx % F);
  dH[i * F + f] += dXN[i * 144 + f];
}

__global__ void k_edge_back(int64_t E, const int* __restrict__ esrc, const float* __restrict__ dXN, float inv_nbar,
                            bf16* __restrict__ dM) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= E * F) return;
  const int64_t e = idx / F;
  const int f = (int)(idx % F);
  dM[e * F + f] = __float2bfloat16_rn(dXN[(int64_t)esrc[e] * 144 + F + f] * inv_nbar);
}

// Reverse of each fluid edge: erev[e] for e = (i -> j) is the edge (j -> i) (the frozen
// fluid neighbour relation is symmetric: |r_i - r_j| < 2h either way); -1 for walls.
__global__ void k_reverse_edges(int64_t E, const int* __restrict__ esrc, const int* __restrict__ enbr,
                                const uint32_t* __restrict__ off, int* __restrict__ erev) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int i = esrc[e], j = enbr[e];
  int r = -1;
  if (j >= 0)
    for (uint32_t e2 = off[j]; e2 < off[j + 1]; ++e2)
      if (enbr[e2] == i) {
        r = (int)e2;
        break;
      }
  erev[e] = r;
}

// Transpose of the gather h_j -> x_ij: dh[j] += sum over edges (i -> j) of dXE[e, fe + f],
// taken over j's own fluid edges (j -> i) through their reverses, in edge order.
__global__ void k_gather_dh(int64_t n, int fe, const uint32_t* __restrict__ off, const int* __restrict__ enbr,
                            const int* __restrict__ erev, const float* __restrict__ dXE, float* __restrict__ dH) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  const int64_t j = idx / F;
  const int f = (int)(idx % F);
  float acc = 0.f;
  for (uint32_t e2 = off[j]; e2 < off[j + 1] && enbr[e2] >= 0; ++e2) {
    const int r = erev[e2];
    if (r >= 0) acc += dXE[(int64_t)r * 80 + fe + f];
  }
  dH[j * F + f] += acc;
}

// dZ0 = bf16(dh * (h0 > 0))
__global__ void k_relu_back(int64_t n, const float* __restrict__ dH, const float* __restrict__ H0,
                            bf16* __restrict__ dZ) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  dZ[idx] = __float2bfloat16_rn(H0[idx] > 0.f ? dH[idx] : 0.f);
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8); b1pow = beta1^t, b2pow = beta2^t
__global__ void k_adam(int count, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1pow, float b2pow) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= count) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  m[o] = b1 * m[o] + (1.f - b1) * g[o];
  v[o] = b2 * v[o] + (1.f - b2) * g[o] * g[o];
  const float mh = m[o] / (1.f - b1pow), vh = v[o] / (1.f - b2pow);
  w[o] -= lr * mh / (sqrtf(vh) + eps);
}

// bf16 copies of the weights: row-major and, per matrix, transposed
__global__ void k_weights_bf16(const float* __restrict__ w, bf16* __restrict__ wb, bf16* __restrict__ wbt) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= kWeights) return;
  int base = 0, l = 0;
  while (l < L_COUNT - 1 && o >= base + c_rows[l] * c_cols[l]) {
    base += c_rows[l] * c_cols[l];
    ++l;
  }
  const int r = (o - base) / c_cols[l], c = (o - base) % c_cols[l];
  const bf16 b = __float2bfloat16_rn(w[o]);
  wb[o] = b;
  wbt[base + c * c_rows[l] + r] = b;
}

// Apply a prediction: v' = v + g Dt_ad + V_S y_v, rho' = rho + rho0 y_rho / 100,
// r' = r + Dt_ad (v + v')/2, d rho/dt = (rho' - rho)/Dt_ad; the tank's clock advances by Dt_ad.
template <int D>
__global__ void k_apply(int64_t n, int4* __restrict__ P, float4* __restrict__ V, const int* __restrict__ inst_of,
                        const Inst* __restrict__ inst, const Ctrl* __restrict__ ctrl, const float* __restrict__ Y,
                        Global* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = inst_of ? inst_of[i] : 0;
  const Inst& I = inst[k];
  const float dt = (float)ctrl[k].dt_ad;
  const float gmag = sqrtf(I.g[0] * I.g[0] + I.g[1] * I.g[1] + I.g[2] * I.g[2]);
  const float vs = gmag > 0.f ? gmag * dt : (float)I.u_ref;
  int4 p = P[i];
  const float4 v = V[i];
  const float* y = Y + i * 16;
  const float vn[3] = {v.x + I.g[0] * dt + vs * y[0], v.y + I.g[1] * dt + vs * y[1],
                       D == 3 ? v.z + I.g[2] * dt + vs * y[2] : 0.f};
  const float drho = I.rho0 * y[D] / S_RHO;
  const float dev = i2f(p.w) + drho;
  const float vo[3] = {v.x, v.y, v.z};
  int q[3] = {p.x, p.y, p.z};
  for (int a = 0; a < D; ++a) q[a] = wrap_coord(q[a] + __float2int_rn(0.5f * dt * (vo[a] + vn[a]) * I.inv_dq), I.period[a]);
  if (!isfinite(dev) || !isfinite(vn[0]) || !isfinite(vn[1])) atomicOr(&g->err, ERR_NAN);
  P[i] = make_int4(q[0], q[1], q[2], f2i(dev));
  V[i] = make_float4(vn[0], vn[1], vn[2], dt > 0.f ? drho / dt : 0.f);
}

__global__ void k_learned_clock(int n_inst, Ctrl* ctrl) {
  for (int k = threadIdx.x; k < n_inst; k += blockDim.x) {
    ctrl[k].t += ctrl[k].dt_ad;
    ctrl[k].tau = ctrl[k].dt_ad;
    ctrl[k].done = 1;
    ctrl[k].dt = 0.0;
  }
}

template <int NO>
size_t dense_smem(int K) {
  // W and two A tiles; at least enough that no more CTAs share an SM than its 512 TMEM
  // columns hold, so a TMEM allocation never waits
  const size_t need = (size_t)dense_w_bytes(NO, K) + 2 * (size_t)dense_tile_bytes(K);
  const size_t per_sm = 233472;                               // shared memory of an SM
  const size_t floor = per_sm / (size_t)(512 / tc::tmem_cols(NO) + 1) + 1;
  return std::max(need, floor);
}

template <int NO>
size_t dw_smem(int K) { return (size_t)kTile * ((NO + 8) + (K + 8)) * sizeof(bf16); }

template <int NO>
void set_smem_attrs() {
  cudaFuncSetAttribute(k_dense<NO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)std::max(dense_smem<NO>(144), dense_smem<NO>(16)));
}

template <int NO>
void set_dw_attrs() {
  cudaFuncSetAttribute(k_dense_dw<NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dw_smem<NO>(144));
}

}  // namespace learned
}  // namespace sph

using namespace sph::learned;

struct sph_learned {
  int dim = 2;
  float* w32 = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  bf16* wb = nullptr;
  bf16* wbt = nullptr;
  int64_t adam_t = 0;
  int fused = 1;                             // inference rounds: 0 layer by layer, 1 warp MMA, 2 tcgen05 pipeline
  int* tc_err = nullptr;                     // the handle's device error word (tensor-core waits)
  // workspace
  int64_t cap_n = 0, cap_e = 0;
  uint32_t* cnt = nullptr;
  uint32_t* off = nullptr;
  uint32_t* scan_tmp = nullptr;
  int* esrc = nullptr;
  int* enbr = nullptr;
  bf16* U = nullptr;
  bf16* XS = nullptr;                        // [E][16] static edge features
  bf16* T = nullptr;                         // [n + 1][80] round input row templates
  int* erev = nullptr;                       // [E] reverse of each fluid edge, -1 for walls
  bf16* XE[ROUNDS] = {nullptr};
  bf16* A1[ROUNDS] = {nullptr};
  bf16* XN[ROUNDS] = {nullptr};
  bf16* A2[ROUNDS] = {nullptr};
  float* Mbuf = nullptr;
  float* H = nullptr;
  float* H0 = nullptr;
  bf16* XD = nullptr;
  bf16* A3 = nullptr;
  float* Y = nullptr;
  float* dH = nullptr;
  float* dXN = nullptr;
  bf16* dYb = nullptr;
  bf16* dZn = nullptr;
  bf16* dM = nullptr;
  bf16* dZe = nullptr;
  float* dXE = nullptr;
  float* partial = nullptr;
  size_t partial_elems = 0;
  double* loss = nullptr;
  int64_t E = 0;
  // saved state for the fallback
  int4* saveP = nullptr;
  float4* saveV = nullptr;
  sph::Ctrl* saveC = nullptr;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

template <typename T>
bool nalloc(sph_learned* L, T** p, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  L->allocs.push_back((void*)*p);
  return true;
}

inline unsigned blocks_for(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

int ensure_workspace(sph_learned* L, int64_t n, int64_t E) {
  if (n <= L->cap_n && E <= L->cap_e) return SPH_OK;
  // grow: free the old workspace (not the weights) and allocate anew
  void* keep[6] = {L->w32, L->m, L->v, L->grad, L->wb, L->wbt};
  std::vector<void*> rest;
  for (void* p : L->allocs) {
    bool k = false;
    for (void* q : keep) k |= (p == q);
    if (k) rest.push_back(p);
    else cudaFree(p);
  }
  L->allocs = rest;
  L->saveC = nullptr;                        // freed above with the rest of the workspace
  n = std::max<int64_t>(n, L->cap_n);
  E = std::max<int64_t>(E, L->cap_e);
  bool ok = nalloc(L, &L->cnt, n) && nalloc(L, &L->off, n + 1) &&
            nalloc(L, &L->scan_tmp, sph::scan_tmp_elems(n)) && nalloc(L, &L->esrc, E) && nalloc(L, &L->enbr, E) && nalloc(L, &L->XS, E * 16) && nalloc(L, &L->erev, E) &&
            nalloc(L, &L->U, n * 16) && nalloc(L, &L->Mbuf, E * F) && nalloc(L, &L->H, n * F) &&
            nalloc(L, &L->H0, n * F) && nalloc(L, &L->XD, n * 80) && nalloc(L, &L->A3, n * 80) &&
            nalloc(L, &L->Y, n * 16) && nalloc(L, &L->dH, n * F) && nalloc(L, &L->dXN, n * 144) &&
            nalloc(L, &L->dYb, n * 16) && nalloc(L, &L->dZn, n * F) && nalloc(L, &L->dM, E * F) &&
            nalloc(L, &L->dZe, std::max(E, n) * F) && nalloc(L, &L->dXE, E * 80) && nalloc(L, &L->loss, 1) &&
            nalloc(L, &L->saveP, n) && nalloc(L, &L->saveV, n) && nalloc(L, &L->T, (n + 1) * 80);
  for (int r = 0; r < ROUNDS && ok; ++r)
    ok = nalloc(L, &L->XE[r], E * 80) && nalloc(L, &L->A1[r], E * 80) && nalloc(L, &L->XN[r], n * 144) &&
         nalloc(L, &L->A2[r], n * 80);
  L->partial_elems = (size_t)((std::max(n, E) + kDwRows - 1) / kDwRows + 1) * 64 * 144;
  ok = ok && nalloc(L, &L->partial, L->partial_elems);
  if (!ok) {
    L->err = "device allocation of the network workspace failed";
    return SPH_E_OOM;
  }
  L->cap_n = n;
  L->cap_e = E;
  // constant columns of the activation buffers (bias 1 and zero padding): no kernel writes
  // them afterwards, so they are set once for every row the workspace holds
  auto consts = [](int64_t rows, int ld, int one, int pad_from, bf16* A) {
    if (rows > 0) k_const_cols<<<blocks_for(rows), 256>>>(rows, ld, one, pad_from, A);
  };
  for (int r = 0; r < ROUNDS; ++r) {
    consts(E, 80, F, F + 1, L->A1[r]);
    consts(n, 144, 2 * F, 2 * F + 1, L->XN[r]);
    consts(n, 80, F, F + 1, L->A2[r]);
  }
  consts(n, 80, F, F + 1, L->XD);
  consts(n, 80, F, F + 1, L->A3);
  if (cudaDeviceSynchronize() != cudaSuccess) {   // before work on the caller's stream uses them
    L->err = "initialising the network workspace failed";
    return SPH_E_CUDA;
  }
  return SPH_OK;
}

template <int NO>
void dense(int64_t M, int K, const bf16* X, int ldx, const bf16* W, float* of, int ldf, int nf, int accum,
           bf16* ob, int ldo, int col0, int nb, int relu, const bf16* mask, int ldm, int* err, cudaStream_t s) {
  if (M == 0) return;
  // K in MMA steps of 16; rows move as 16-byte pieces, results as 16-byte pieces: strides
  // and column ranges must allow it
  if (K % 16 || K > 144 || ldx % 8 || (of && (ldf % 4 || nf % 4)) || (ob && (ldo % 8 || col0 % 8 || nb % 8)) ||
      (mask && ldm % 2)) {
    std::fprintf(stderr, "sph_learned: dense layer with unaligned shape\n");
    return;
  }
  const int64_t tiles = (M + 127) / 128;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, 152 * 8);
  k_dense<NO><<<grid, 128, dense_smem<NO>(K), s>>>(M, K, X, ldx, W, of, ldf, nf, accum, ob, ldo, col0, nb, relu,
                                                   mask, ldm, err);
}

// grad[layer] += dY^T X over M rows
template <int NO>
void dense_dw(sph_learned* L, int layer, int64_t M, int K, const bf16* dY, int ldy, const bf16* X, int ldx,
              cudaStream_t s) {
  if (M == 0) return;
  const int blocks = (int)((M + kDwRows - 1) / kDwRows);
  k_dense_dw<NO><<<blocks, 128, dw_smem<NO>(K), s>>>(M, K, dY, ldy, X, ldx, L->partial);
  const int count = NO * K;
  k_reduce_partials<<<blocks_for(count), 256, 0, s>>>(blocks, count, L->partial, L->grad + w_offset(layer));
}

const bf16* Wl(const sph_learned* L, int l) { return L->wb + w_offset(l); }
const bf16* WTl(const sph_learned* L, int l) { return L->wbt + w_offset(l); }

// Graph and features of the handle's current (post density re-initialisation) state.
int build_inputs(sph_handle* h, sph_learned* L, cudaStream_t s) {
  const sph::Buffers& b = h->b;
  const int64_t n = b.n;
  // edge count first (host needs E to size the workspace)
  if (ensure_workspace(L, n, std::max<int64_t>(L->cap_e, 1)) != SPH_OK) return SPH_E_OOM;
  k_edge_count<<<blocks_for(n), 256, 0, s>>>(n, b.nbc, L->cnt);
  int64_t dummy = 0;
  sph::scan_exclusive(L->cnt, L->off, n, L->scan_tmp, s, &dummy);
  uint32_t E32 = 0;
  if (cudaMemcpyAsync(&E32, L->off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return SPH_E_CUDA;
  }
  const int64_t E = E32;
  if (E > L->cap_e) {
    if (ensure_workspace(L, n, E) != SPH_OK) return SPH_E_OOM;
    k_edge_count<<<blocks_for(n), 256, 0, s>>>(n, b.nbc, L->cnt);
    sph::scan_exclusive(L->cnt, L->off, n, L->scan_tmp, s, &dummy);
  }
  L->E = E;
  if (b.dim == 2) {
    k_node_features<2><<<blocks_for(n), 256, 0, s>>>(n, b.PS, b.VS, b.inst_of, b.inst, b.ctrl, b.nbr, b.nbc, L->off,
                                                     L->esrc, L->enbr, L->U);
    if (E > 0)
      k_edge_features<2><<<blocks_for(E), 256, 0, s>>>(E, b.PS, b.VS, b.inst_of, b.inst, L->esrc, L->enbr, b.WP,
                                                     L->XS);
  } else {
    k_node_features<3><<<blocks_for(n), 256, 0, s>>>(n, b.PS, b.VS, b.inst_of, b.inst, b.ctrl, b.nbr, b.nbc, L->off,
                                                     L->esrc, L->enbr, L->U);
    if (E > 0)
      k_edge_features<3><<<blocks_for(E), 256, 0, s>>>(E, b.PS, b.VS, b.inst_of, b.inst, L->esrc, L->enbr, b.WP,
                                                     L->XS);
  }
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}

// train: keep every round's edge rows and activations for the backward pass; otherwise
// (inference) the edge network of each round runs fused when the network allows it.
void forward(sph_handle* h, sph_learned* L, cudaStream_t s, bool train) {
  L->tc_err = &h->b.glob->err;
  const int64_t n = h->b.n, E = L->E;
  const int d = h->b.dim, fe = 2 * d + 3;
  const float inv_nbar = 1.0f / nbar(d);
  const bool fused = L->fused == 1 && !train;
  const bool piped = L->fused == 2 && !train;
  // encoder: H = relu(U W_enc^T); H0 keeps h0 for the encoder's backward
  dense<64>(n, 16, L->U, 16, Wl(L, L_ENC), L->H, F, F, 0, nullptr, 0, 0, 0, 1, nullptr, 0, L->tc_err, s);
  if (train) cudaMemcpyAsync(L->H0, L->H, sizeof(float) * n * F, cudaMemcpyDeviceToDevice, s);
  for (int r = 0; r < ROUNDS; ++r) {
    if (fused) {
      const int64_t chunks = (n + kFuseNodes - 1) / kFuseNodes;
      int per_sm = 1, sms = 1, dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      auto kern = d == 2 ? k_edge_round_fused<7> : k_edge_round_fused<9>;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFuseWarps * 32, fused_smem());
      const unsigned grid = (unsigned)std::min<int64_t>((chunks + kFuseWarps - 1) / kFuseWarps,
                                                        (int64_t)std::max(per_sm, 1) * sms);
      // node states ping-pong between H and H0 (H0 is only kept for training's backward)
      float* hin = (r & 1) ? L->H0 : L->H;
      float* hout = (r & 1) ? L->H : L->H0;
      if (n > 0)
        kern<<<grid, kFuseWarps * 32, fused_smem(), s>>>(n, L->off, L->XS, L->enbr, hin, Wl(L, L_E1), Wl(L, L_E2),
                                                         Wl(L, L_N1), Wl(L, L_N2), inv_nbar, L->XN[r], hout);
    } else if (piped) {
      auto tmpl = d == 2 ? k_node_templates<7> : k_node_templates<9>;
      tmpl<<<blocks_for((n + 1) * 10 + n * 8), 256, 0, s>>>(n, L->H, L->T, L->XN[r]);
      if (n > 0) {
        int sms = 1, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // runs of equal node counts, a whole number of them per CTA where possible
        const int64_t slots = 2 * (int64_t)sms;
        const int64_t per = (n + slots * kWsRun - 1) / (slots * kWsRun);
        const int run = (int)std::max<int64_t>(1, (n + slots * per - 1) / (slots * per));
        const int64_t runs = (n + run - 1) / run;
        const unsigned grid = (unsigned)std::min<int64_t>(runs, slots);
        auto kern = d == 2 ? k_edge_round_ws<7> : k_edge_round_ws<9>;
        kern<<<grid, kWsThreads, ws_smem(), s>>>(n, run, L->off, L->XS, L->enbr, L->T, Wl(L, L_E1), Wl(L, L_E2),
                                                 inv_nbar, L->XN[r], L->tc_err);
      }
      dense<64>(n, 144, L->XN[r], 144, Wl(L, L_N1), nullptr, 0, 0, 0, L->A2[r], 80, 0, F, 1, nullptr, 0, L->tc_err, s);
      dense<64>(n, 80, L->A2[r], 80, Wl(L, L_N2), L->H, F, F, 1, nullptr, 0, 0, 0, 0, nullptr, 0, L->tc_err, s);
    } else {
      if (E > 0) k_edge_rows<<<blocks_for(E * 10), 256, 0, s>>>(E, fe, L->XS, L->enbr, L->H, L->XE[r]);
      dense<64>(E, 80, L->XE[r], 80, Wl(L, L_E1), nullptr, 0, 0, 0, L->A1[r], 80, 0, F, 1, nullptr, 0, L->tc_err, s);
      dense<64>(E, 80, L->A1[r], 80, Wl(L, L_E2), L->Mbuf, F, F, 0, nullptr, 0, 0, 0, 0, nullptr, 0, L->tc_err, s);
      k_segsum<<<blocks_for(n * F), 256, 0, s>>>(n, L->off, L->Mbuf, L->H, inv_nbar, L->XN[r]);
      dense<64>(n, 144, L->XN[r], 144, Wl(L, L_N1), nullptr, 0, 0, 0, L->A2[r], 80, 0, F, 1, nullptr, 0, L->tc_err, s);
      dense<64>(n, 80, L->A2[r], 80, Wl(L, L_N2), L->H, F, F, 1, nullptr, 0, 0, 0, 0, nullptr, 0, L->tc_err, s);
    }
  }
  // the fused rounds leave the final node states in H0 after an odd number of rounds
  const float* hfin = (fused && (ROUNDS & 1)) ? L->H0 : L->H;
  k_rows_bf16<<<blocks_for(n * F), 256, 0, s>>>(n, F, hfin, F, L->XD, 80);
  dense<64>(n, 80, L->XD, 80, Wl(L, L_D1), nullptr, 0, 0, 0, L->A3, 80, 0, F, 1, nullptr, 0, L->tc_err, s);
  dense<16>(n, 80, L->A3, 80, Wl(L, L_D2), L->Y, 16, 16, 0, nullptr, 0, 0, 0, 0, nullptr, 0, L->tc_err, s);
}

void backward(sph_handle* h, sph_learned* L, cudaStream_t s) {
  L->tc_err = &h->b.glob->err;
  const int64_t n = h->b.n, E = L->E;
  const int d = h->b.dim, fe = 2 * d + 3;
  const float inv_nbar = 1.0f / nbar(d);
  cudaMemsetAsync(L->grad, 0, sizeof(float) * kWeights, s);
  if (E > 0) k_reverse_edges<<<blocks_for(E), 256, 0, s>>>(E, L->esrc, L->enbr, L->off, L->erev);
  // decoder
  dense_dw<16>(L, L_D2, n, 80, L->dYb, 16, L->A3, 80, s);
  dense<80>(n, 16, L->dYb, 16, WTl(L, L_D2), nullptr, 0, 0, 0, L->dZn, F, 0, F, 0, L->A3, 80, L->tc_err, s);
  dense_dw<64>(L, L_D1, n, 80, L->dZn, F, L->XD, 80, s);
  dense<80>(n, 64, L->dZn, F, WTl(L, L_D1), L->dH, F, F, 0, nullptr, 0, 0, 0, 0, nullptr, 0, L->tc_err, s);
  for (int r = ROUNDS - 1; r >= 0; --r) {
    // h_new = h + W_n2 [relu(W_n1 XN), 1]
    k_rows_bf16<<<blocks_for(n * F), 256, 0, s>>>(n, F, L->dH, F, L->dZn, F);
    dense_dw<64>(L, L_N2, n, 80, L->dZn, F, L->A2[r], 80, s);
    bf16* dZ2 = L->dZe;   // reuse the edge buffer (E >= n)
    dense<80>(n, 64, L->dZn, F, WTl(L, L_N2), nullptr, 0, 0, 0, dZ2, F, 0, F, 0, L->A2[r], 80, L->tc_err, s);
    dense_dw<64>(L, L_N1, n, 144, dZ2, F, L->XN[r], 144, s);
    dense<144>(n, 64, dZ2, F, WTl(L, L_N1), L->dXN, 144, 144, 0, nullptr, 0, 0, 0, 0, nullptr, 0, L->tc_err, s);
    k_node_back<<<blocks_for(n * F), 256, 0, s>>>(n, L->dXN, L->dH);
    if (E > 0) k_edge_back<<<blocks_for(E * F), 256, 0, s>>>(E, L->esrc, L->dXN, inv_nbar, L->dM);
    dense_dw<64>(L, L_E2, E, 80, L->dM, F, L->A1[r], 80, s);
    dense<80>(E, 64, L->dM, F, WTl(L, L_E2), nullptr, 0, 0, 0, L->dZe, F, 0, F, 0, L->A1[r], 80, L->tc_err, s);
    dense_dw<64>(L, L_E1, E, 80, L->dZe, F, L->XE[r], 80, s);
    dense<80>(E, 64, L->dZe, F, WTl(L, L_E1), L->dXE, 80, 80, 0, nullptr, 0, 0, 0, 0, nullptr, 0, L->tc_err, s);
    if (E > 0) k_gather_dh<<<blocks_for(n * F), 256, 0, s>>>(n, fe, L->off, L->enbr, L->erev, L->dXE, L->dH);
  }
  k_relu_back<<<blocks_for(n * F), 256, 0, s>>>(n, L->dH, L->H0, L->dZn);
  dense_dw<64>(L, L_ENC, n, 16, L->dZn, F, L->U, 16, s);
}

}  // namespace

// ------------------------------------------------------------------ C ABI
namespace {

__global__ void k_export_y(int64_t n, int dout, const float* __restrict__ Y, const int* __restrict__ id,
                           double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t row = id[i];
  for (int c = 0; c < dout; ++c) y[row * dout + c] = (double)Y[i * 16 + c];
}

// Memory the current device can address directly (its own or managed); device memory
// of another GPU counts as not addressable (see foreign_ptr).
bool device_ptr(const void* p) {
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

// Device memory of a GPU other than the current one: rejected by the entry points, since
// the kernels run on the current device.
bool foreign_ptr(const void* p) {
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

int lfail(sph_learned* L, int code, const char* msg) {
  if (L) L->err = msg;
  return code;
}

void upload_weights_bf16(sph_learned* L, cudaStream_t s) {
  k_weights_bf16<<<blocks_for(kWeights), 256, 0, s>>>(L->w32, L->wb, L->wbt);
}

int ready(sph_handle* h, sph_learned* L, void* stream) {
  if (!h || !L) return SPH_E_INVALID;
  if (h->b.dim != L->dim) return lfail(L, SPH_E_INVALID, "network and handle dimensions differ");
  if (!h->cells_valid) return lfail(L, SPH_E_INVALID, "run sph_build_cells and sph_advection_step first");
  const int r = sph_debug_check(h, (cudaStream_t)stream);
  if (r != SPH_OK) return lfail(L, r, "neighbour table check failed (SPH_FLAG_DEBUG_BOUNDS)");
  return SPH_OK;
}

}  // namespace

extern "C" {

int sph_learned_weight_count(int64_t* count) {
  if (!count) return SPH_E_INVALID;
  *count = kWeights;
  return SPH_OK;
}

const char* sph_learned_last_error(const sph_learned* L) { return L ? L->err.c_str() : "null network"; }

void sph_learned_destroy(sph_learned* L) {
  if (!L) return;
  for (void* p : L->allocs) cudaFree(p);
  delete L;
}

int sph_learned_create(int32_t dim, const float* weights, sph_learned** out) {
  if (!out || (dim != 2 && dim != 3)) return SPH_E_INVALID;
  sph_learned* L = new sph_learned();
  *out = L;
  L->dim = dim;
  if (!nalloc(L, &L->w32, kWeights) || !nalloc(L, &L->m, kWeights) || !nalloc(L, &L->v, kWeights) ||
      !nalloc(L, &L->grad, kWeights) || !nalloc(L, &L->wb, kWeights) || !nalloc(L, &L->wbt, kWeights))
    return lfail(L, SPH_E_OOM, "device allocation of the weights failed");
  cudaFuncSetAttribute(k_edge_round_fused<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem());
  cudaFuncSetAttribute(k_edge_round_fused<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem());
  cudaFuncSetAttribute(k_edge_round_ws<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem());
  cudaFuncSetAttribute(k_edge_round_ws<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem());
  set_smem_attrs<16>();
  set_smem_attrs<64>();
  set_smem_attrs<80>();
  set_smem_attrs<144>();
  set_dw_attrs<16>();
  set_dw_attrs<64>();
  cudaMemset(L->m, 0, sizeof(float) * kWeights);
  cudaMemset(L->v, 0, sizeof(float) * kWeights);
  cudaMemset(L->w32, 0, sizeof(float) * kWeights);
  if (weights && cudaMemcpy(L->w32, weights, sizeof(float) * kWeights, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return lfail(L, SPH_E_CUDA, "copy of the weights failed");
  }
  upload_weights_bf16(L, 0);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return lfail(L, SPH_E_CUDA, "network set-up failed");
  }
  return SPH_OK;
}

int sph_learned_set_weights(sph_learned* L, const float* w) {
  if (!L || !w) return SPH_E_INVALID;
  if (cudaMemcpy(L->w32, w, sizeof(float) * kWeights, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return lfail(L, SPH_E_CUDA, "copy of the weights failed");
  }
  cudaMemset(L->m, 0, sizeof(float) * kWeights);
  cudaMemset(L->v, 0, sizeof(float) * kWeights);
  L->adam_t = 0;
  upload_weights_bf16(L, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}

int sph_learned_get_weights(sph_learned* L, float* w) {
  if (!L || !w) return SPH_E_INVALID;
  if (cudaMemcpy(w, L->w32, sizeof(float) * kWeights, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return lfail(L, SPH_E_CUDA, "copy of the weights failed");
  }
  return SPH_OK;
}

int sph_learned_set_fused(sph_learned* L, int32_t enabled) {
  if (!L) return SPH_E_INVALID;
  if (enabled < 0 || enabled > 2) return SPH_E_INVALID;
  L->fused = enabled;
  return SPH_OK;
}

int sph_learned_predict(sph_handle* h, sph_learned* L, double* y, void* stream) {
  int r = ready(h, L, stream);
  if (r != SPH_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  r = build_inputs(h, L, s);
  if (r != SPH_OK) return lfail(L, r, "building the network inputs failed");
  if (foreign_ptr(y)) return lfail(L, SPH_E_INVALID, "y lives on another device");
  forward(h, L, s, false);
  if (y) {
    const int dout = h->b.dim + 1;
    const bool dev = device_ptr(y);
    double* tgt = dev ? y : h->stage;
    k_export_y<<<blocks_for(h->b.n), 256, 0, s>>>(h->b.n, dout, L->Y, h->b.id, tgt);
    if (!dev && cudaMemcpyAsync(y, tgt, sizeof(double) * h->b.n * dout, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      cudaGetLastError();
      return lfail(L, SPH_E_CUDA, "copy of the prediction failed");
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return lfail(L, SPH_E_CUDA, "network forward pass failed");
  }
  return SPH_OK;
}

int sph_learned_train_step(sph_handle* h, sph_learned* L, const double* target, double lr, double* loss_out,
                           float* grad_out, void* stream) {
  int r = ready(h, L, stream);
  if (r != SPH_OK) return r;
  if (!target) return lfail(L, SPH_E_INVALID, "target is required");
  if (foreign_ptr(target)) return lfail(L, SPH_E_INVALID, "target lives on another device");
  cudaStream_t s = (cudaStream_t)stream;
  r = build_inputs(h, L, s);
  if (r != SPH_OK) return lfail(L, r, "building the network inputs failed");
  forward(h, L, s, true);
  const int64_t n = h->b.n;
  const int dout = h->b.dim + 1;
  const double* T = target;
  if (!device_ptr(target)) {
    if (cudaMemcpyAsync(h->stage, target, sizeof(double) * n * dout, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return lfail(L, SPH_E_CUDA, "copy of the target failed");
    }
    T = h->stage;
  }
  cudaMemsetAsync(L->loss, 0, sizeof(double), s);
  k_loss<<<blocks_for(n), 256, 0, s>>>(n, dout, L->Y, T, h->b.id, L->dYb, L->loss);
  backward(h, L, s);
  if (lr > 0.0) {
    ++L->adam_t;
    const float b1pow = (float)std::pow(0.9, (double)L->adam_t), b2pow = (float)std::pow(0.999, (double)L->adam_t);
    k_adam<<<blocks_for(kWeights), 256, 0, s>>>(kWeights, L->w32, L->m, L->v, L->grad, (float)lr, b1pow, b2pow);
    upload_weights_bf16(L, s);
  }
  double loss = 0.0;
  cudaMemcpyAsync(&loss, L->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (grad_out) cudaMemcpyAsync(grad_out, L->grad, sizeof(float) * kWeights, cudaMemcpyDefault, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return lfail(L, SPH_E_CUDA, "training step failed");
  }
  if (loss_out) *loss_out = loss;
  return SPH_OK;
}

int sph_learned_step(sph_handle* h, sph_learned* L, double max_mean_rho_dev, double max_energy_drift,
                     int32_t* used_learned, void* stream) {
  if (!h || !L) return SPH_E_INVALID;
  if (h->b.dim != L->dim) return lfail(L, SPH_E_INVALID, "network and handle dimensions differ");
  cudaStream_t s = (cudaStream_t)stream;
  int r = sph_build_cells(h, stream);
  if (r == SPH_OK) r = sph_advection_step(h, nullptr, stream);
  if (r != SPH_OK) return r;
  const int K = h->b.n_inst;
  std::vector<sph_diag> d0(K), d1(K);
  r = sph_diagnostics(h, d0.data(), stream);
  if (r != SPH_OK) return r;
  const int64_t n = h->b.n;
  r = build_inputs(h, L, s);
  if (r != SPH_OK) return lfail(L, r, "building the network inputs failed");
  if (!L->saveC && !nalloc(L, &L->saveC, K)) return lfail(L, SPH_E_OOM, "allocation failed");
  cudaMemcpyAsync(L->saveP, h->b.PS, sizeof(int4) * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(L->saveV, h->b.VS, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(L->saveC, h->b.ctrl, sizeof(sph::Ctrl) * K, cudaMemcpyDeviceToDevice, s);
  forward(h, L, s, false);
  if (h->b.dim == 2)
    k_apply<2><<<blocks_for(n), 256, 0, s>>>(n, h->b.PS, h->b.VS, h->b.inst_of, h->b.inst, h->b.ctrl, L->Y, h->b.glob);
  else
    k_apply<3><<<blocks_for(n), 256, 0, s>>>(n, h->b.PS, h->b.VS, h->b.inst_of, h->b.inst, h->b.ctrl, L->Y, h->b.glob);
  k_learned_clock<<<1, 256, 0, s>>>(K, h->b.ctrl);
  sph::launch_vmax(h->b, s, &h->launches);
  h->cells_valid = false;
  r = sph_diagnostics(h, d1.data(), stream);
  bool ok = (r == SPH_OK);
  for (int k = 0; k < K && ok; ++k) {
    const double drift = std::fabs(d1[k].energy - d0[k].energy) / std::max(std::fabs(d0[k].energy), 1e-300);
    if (!(d1[k].mean_rho_dev <= max_mean_rho_dev) || !(drift <= max_energy_drift)) ok = false;
  }
  if (used_learned) *used_learned = ok ? 1 : 0;
  if (ok) return SPH_OK;
  // fall back: restore the step's start and run the acoustic substeps
  h->err.clear();
  cudaMemsetAsync(h->b.glob, 0, sizeof(int), s);                    // clear error bits of the trial
  cudaMemcpyAsync(h->b.PS, L->saveP, sizeof(int4) * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(h->b.VS, L->saveV, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(h->b.ctrl, L->saveC, sizeof(sph::Ctrl) * K, cudaMemcpyDeviceToDevice, s);
  h->cells_valid = true;
  for (int guard = 0;; ++guard) {
    int32_t done = 0;
    r = sph_acoustic_substep(h, &done, nullptr, stream);
    if (r != SPH_OK) return r;
    if (done) break;
    if (guard > 1000000) return SPH_E_UNSTABLE;
  }
  return SPH_OK;
}

}  // extern "C"

