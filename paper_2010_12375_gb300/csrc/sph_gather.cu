// Gather ceiling of the acoustic-substep kernels (a diagnostic; the paper has no
// counterpart). The kernel below walks the frozen neighbour table exactly as the pressure
// relaxation does -- one thread per particle, one quad of four slots per 16-byte index
// load with the next quad in flight, the eight 16-byte neighbour records of a quad
// (position + velocity) gathered together, then the wall slots -- but does no pair
// arithmetic: it only folds the gathered words into one value so the loads stay live.
// Its time is what gathering the neighbour records in this layout costs by itself on the
// device, a floor for any kernel that gathers them the same way. It runs in the launch form
// of the pressure relaxation: per particle, or in the row-task form.
#include "sph_kernels.h"

namespace sph {

namespace {

constexpr int kGatherBlock = 128;

__device__ __forceinline__ unsigned fold(const int4& a, const float4& b) {
  return (unsigned)(a.x ^ a.y ^ a.z ^ a.w) ^ __float_as_uint(b.x) ^ __float_as_uint(b.y) ^
         __float_as_uint(b.z) ^ __float_as_uint(b.w);
}

// The walk of particle i's row (valid lanes only); returns the folded words.
__device__ __forceinline__ unsigned walk_particle(int64_t i, int64_t n, const int4* __restrict__ PS,
                                                  const float4* __restrict__ VS, const int* __restrict__ nbr,
                                                  const uint32_t* __restrict__ nbc, const int4* __restrict__ WP,
                                                  const float4* __restrict__ WN) {
  unsigned acc = 0u;
  const uint32_t cnt = nbc[i];
  const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
  const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
  const int nq = (nf + 3) >> 2;
  int4 cur = nq ? nb4[i] : make_int4(0, 0, 0, 0);
  for (int q = 0; q < nq; ++q) {
    int4 nxt = cur;
    if (q + 1 < nq) nxt = nb4[(int64_t)(q + 1) * n + i];
    const int s = q << 2;
    const int j0 = cur.x;
    const int j1 = s + 1 < nf ? cur.y : (int)i;
    const int j2 = s + 2 < nf ? cur.z : (int)i;
    const int j3 = s + 3 < nf ? cur.w : (int)i;
    const int4 p0 = PS[j0], p1 = PS[j1], p2 = PS[j2], p3 = PS[j3];
    const float4 v0 = VS[j0], v1 = VS[j1], v2 = VS[j2], v3 = VS[j3];
    acc ^= fold(p0, v0) ^ fold(p1, v1) ^ fold(p2, v2) ^ fold(p3, v3);
    cur = nxt;
  }
  if (nw) {
    const int q0 = wall_slot0(nf) >> 2, nwq = (nw + 3) >> 2;
    for (int q = 0; q < nwq; ++q) {
      const int4 c = nb4[(int64_t)(q0 + q) * n + i];
      const int s = q << 2;
      const int w1 = s + 1 < nw ? c.y : c.x, w2 = s + 2 < nw ? c.z : c.x, w3 = s + 3 < nw ? c.w : c.x;
      acc ^= fold(WP[c.x], WN[c.x]) ^ fold(WP[w1], WN[w1]) ^ fold(WP[w2], WN[w2]) ^ fold(WP[w3], WN[w3]);
    }
  }
  return acc;
}

__device__ __forceinline__ void sink_warp(unsigned acc, unsigned* sink) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc == 0x9e3779b9u) atomicXor(sink, acc);   // practically never taken
}

__global__ void __launch_bounds__(kGatherBlock)
k_gather_ceiling(int64_t n, const int4* __restrict__ PS, const float4* __restrict__ VS,
                 const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                 const int4* __restrict__ WP, const float4* __restrict__ WN, unsigned* __restrict__ sink) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  sink_warp(i < n ? walk_particle(i, n, PS, VS, nbr, nbc, WP, WN) : 0u, sink);
}

// The same walk in the row-task launch form of the relaxations (one resident block of
// kRowWarps warps an SM, 32-particle row pieces from the block's queue, runs of kRowWarps
// pieces numbered b, b + gridDim.x, ...): the floor for the row-task kernels.
__global__ void __launch_bounds__(kRowBlock, 1)
k_gather_ceiling_rows(int64_t n, const int4* __restrict__ PS, const float4* __restrict__ VS,
                      const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                      const int4* __restrict__ WP, const float4* __restrict__ WN, unsigned* __restrict__ sink,
                      const int2* __restrict__ row_task, const uint32_t* __restrict__ row_total,
                      int64_t row_task_cap) {
  __shared__ int queue;
  if (threadIdx.x == 0) queue = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long pieces = min((long long)*row_total, (long long)row_task_cap);
  unsigned acc = 0u;
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(&queue, 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    const long long t = ((long long)blockIdx.x + (long long)gridDim.x * (q / kRowWarps)) * kRowWarps + q % kRowWarps;
    if (t >= pieces) break;
    const int2 piece = row_task[t];
    if (lane < piece.y) acc ^= walk_particle((int64_t)piece.x + lane, n, PS, VS, nbr, nbc, WP, WN);
  }
  sink_warp(acc, sink);
}

}  // namespace

bool gather_rows(const Buffers& b) { return row_form(b.cfg.pr_block) && b.row_task && !b.geo; }

void launch_gather_ceiling(const Buffers& b, unsigned* sink, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  if (gather_rows(b)) {                      // the pressure relaxation runs in the row-task form
    if (!*b.rows_valid) {
      launch_row_tasks(b, s, launches);
      *b.rows_valid = true;
    }
    k_gather_ceiling_rows<<<b.n_sm, kRowBlock, 0, s>>>(b.n, b.PS, b.VS, b.nbr, b.nbc, b.nw ? b.WP : nullptr,
                                                       b.nw ? b.WN : nullptr, sink, b.row_task,
                                                       b.row_off + b.n_rows, b.row_task_cap);
    ++*launches;
    return;
  }
  const unsigned grid = (unsigned)((b.n + kGatherBlock - 1) / kGatherBlock);
  k_gather_ceiling<<<grid, kGatherBlock, 0, s>>>(b.n, b.PS, b.VS, b.nbr, b.nbc, b.nw ? b.WP : nullptr,
                                                 b.nw ? b.WN : nullptr, sink);
  ++*launches;
}

}  // namespace sph
