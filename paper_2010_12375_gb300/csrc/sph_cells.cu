// Configuration update of the WCSPH hot path (cell-linked list, paper Sec. 6.2
// mesh_cell_linked_list, refreshed once per advection step as Sec. 2.4 fixes):
//   hash      particle -> search cell (integer: q >> (bits - 1) per axis, i.e. cells of
//             half the 2h position cell, about h; flattened x fastest)
//   sort      counting sort on the cell digit (a one-digit radix sort with radix =
//             number of cells), then each particle's rank among its cell mates by
//             caller id, which makes the order the unique (cell, id) order,
//             independent of history
//   offsets   exclusive scan of the cell counts
//   reorder   the 32-byte particle records moved to their (cell, id) slots
//   neighbours frozen set {j != i : |r_i - r_j| < 2h}, quad-interleaved ELL rows; the
//             search visits the 5^D cells around a particle clipped to its 2h sphere
//             (rows whose slab lies at >= 2h are skipped, row runs cut to the
//             sphere's chord), about 42 % of the candidates of a 3^D scan of 2h cells
#include <cstdio>

#include "sph_kernels.h"

namespace sph {

namespace {

constexpr int kBlock = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

inline unsigned grid_for(int64_t n, int block = kBlock) {
  return (unsigned)((n + block - 1) / block);
}

__device__ __forceinline__ void raise_error(Global* g, int bit, long long idx) {
  int old = atomicOr(&g->err, bit);
  if (old == 0) g->bad_index = idx;
}

// ---------------------------------------------------------------- scan ---------------
// Block-level exclusive scan of kScanTile elements; block totals to `sums`.
__global__ void k_scan_tile(const uint32_t* in, uint32_t* out,   // may alias (in-place)
                            int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t local = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + k;
    v[k] = idx < n ? in[idx] : 0u;
    local += v[k];
  }
  // inclusive scan of per-thread totals inside the warp
  unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (unsigned)o) wi += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;   // exclusive warp offsets
    if (lane == 31 && sums) sums[blockIdx.x] = wi;           // block total
  }
  __syncthreads();
  uint32_t run = warp_tot[warp] + incl - local;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + k;
    if (idx < n) out[idx] = run;
    run += v[k];
  }
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ offs) {
  int64_t idx = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  uint32_t add = offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t j = idx + (int64_t)k * kScanThreads;
    if (j < n) out[j] += add;
  }
}

__global__ void k_scan_total(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n) {
  out[n] = n ? out[n - 1] + in[n - 1] : 0u;
}

}  // namespace

size_t scan_tmp_elems(int64_t n) {
  size_t total = 0;
  int64_t m = n;
  while (m > kScanTile) {
    m = (m + kScanTile - 1) / kScanTile;
    total += (size_t)m;
  }
  return total + 1;
}

static void scan_rec(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s,
                     int64_t* launches) {
  int64_t blocks = (n + kScanTile - 1) / kScanTile;
  if (blocks <= 1) {
    k_scan_tile<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    ++*launches;
    return;
  }
  uint32_t* sums = tmp;
  k_scan_tile<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, sums);
  scan_rec(sums, sums, blocks, tmp + blocks, s, launches);
  k_scan_add<<<(unsigned)blocks, kScanThreads, 0, s>>>(out, n, sums);
  *launches += 2;
}

// Exclusive scan of in[0..n) into out[0..n], out[n] = total.
void scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s,
                    int64_t* launches) {
  if (n > 0) scan_rec(in, out, n, tmp, s, launches);
  k_scan_total<<<1, 1, 0, s>>>(in, out, n);
  ++*launches;
}

namespace {

// ---------------------------------------------------------------- hash ---------------
template <int D>
__global__ void k_hash(int64_t n, const int4* __restrict__ P, const int* __restrict__ inst_of,
                       const Inst* __restrict__ inst, uint32_t* __restrict__ cell,
                       uint32_t* __restrict__ count, uint32_t* __restrict__ rank, Global* g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  int4 p = P[i];
  int q[3] = {p.x, p.y, p.z};
  long long c = 0, stride = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int ca = q[a] >> I.sbits;                       // search cell: half a cell per axis
    if (ca < 0 || ca >= I.scell[a]) {
      raise_error(g, ERR_DOMAIN, i);
      ca = ca < 0 ? 0 : I.scell[a] - 1;
    }
    c += (long long)ca * stride;
    stride *= I.scell[a];
  }
  c += I.cell_base;
  cell[i] = (uint32_t)c;
  rank[i] = atomicAdd(&count[c], 1u);
}

__global__ void k_scatter(int64_t n, const uint32_t* __restrict__ cell, const uint32_t* __restrict__ rank,
                          const uint32_t* __restrict__ start, const int* __restrict__ id,
                          int* __restrict__ key, int* __restrict__ src) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t d = start[cell[i]] + rank[i];
  key[d] = id[i];
  src[d] = (int)i;
}

// Final slot of every particle: the counting sort left each cell's particles in arbitrary
// order; a particle's place within its cell is the number of cell mates with a smaller id,
// which makes the order the unique (cell, id) order. One thread per particle (cells hold
// a few particles), instead of one per cell.
__global__ void k_cell_rank(int64_t n, const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
                            const int* __restrict__ key, const int* __restrict__ src, uint32_t* __restrict__ dst) {
  int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const uint32_t c = cell[src[d]];
  const uint32_t b = start[c], e = start[c + 1];
  const int k = key[d];
  uint32_t r = 0;
  for (uint32_t m = b; m < e; ++m) r += key[m] < k ? 1u : 0u;
  dst[d] = b + r;
}

// Records moved to their final slots (writes stay within each cell's slot range); the
// ids in the new order go to id_out.
__global__ void k_reorder(int64_t n, const int* __restrict__ src, const uint32_t* __restrict__ dst,
                          const int* __restrict__ key, const int4* __restrict__ Pin,
                          const float4* __restrict__ Vin, int4* __restrict__ Pout,
                          float4* __restrict__ Vout, const float* __restrict__ min,
                          float* __restrict__ mout, int* __restrict__ id_out) {
  int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const int s = src[d];
  const uint32_t t = dst[d];
  Pout[t] = Pin[s];
  Vout[t] = Vin[s];
  id_out[t] = key[d];
  if (min) mout[t] = min[s];
}

__global__ void k_copy_back(int64_t n, const int4* __restrict__ Pin, const float4* __restrict__ Vin,
                            const int* __restrict__ key, int4* __restrict__ Pout,
                            float4* __restrict__ Vout, int* __restrict__ id,
                            const float* __restrict__ min, float* __restrict__ mout) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Pout[i] = Pin[i];
  Vout[i] = Vin[i];
  id[i] = key[i];
  if (min) mout[i] = min[i];
}

// ---------------------------------------------------------------- neighbours ---------
__device__ __forceinline__ int wrap_cell(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// Distance (quanta) from a point at offset o inside its search cell (width S) to the
// slab of the cell d rows away; exact integers below 2^23, so exact in FP32.
__device__ __forceinline__ float slab_gap(int d, float o, float S) {
  return d > 0 ? (float)d * S - o : (d < 0 ? o + (float)(-d - 1) * S + 1.0f : 0.0f);
}

// Flattened search cell of a particle (clamped to its tank's grid).
template <int D>
__device__ __forceinline__ long long search_cell(const Inst& I, const int4& p) {
  const int sb = I.sbits;
  const int cx = min(max(p.x >> sb, 0), I.scell[0] - 1);
  const int cy = min(max(p.y >> sb, 0), I.scell[1] - 1);
  const int cz = D == 3 ? min(max(p.z >> sb, 0), I.scell[2] - 1) : 0;
  return I.cell_base + ((long long)cz * I.scell[1] + cy) * I.scell[0] + cx;
}

// Visit the search-cell runs that can hold a neighbour of the particle at p: for every
// row (dy, dz) in [-2, 2]^(D-1) whose slab lies closer than 2h, the x cells that meet the
// sphere's chord in that slab. Within a row the cells of a run are one contiguous slot
// range; a periodic x axis splits a run that crosses the edge into two. The row test and
// the chord are evaluated in FP32 against R2 (1 + 2^-20), a margin above every rounding
// error of the squares, so they only ever err towards visiting more: a particle j in a
// skipped row or cell has sum (q_i - q_j)^2 >= R2 and is not a neighbour.
template <int D, bool PER, typename F>
__device__ __forceinline__ void for_neighbour_runs(const Inst& I, const int4& p,
                                                   const uint32_t* __restrict__ start, F&& visit) {
  const int sb = I.sbits;
  const float S = (float)(1 << sb);
  const int nx = I.scell[0], ny = I.scell[1], nz = D == 3 ? I.scell[2] : 1;
  const int cy = min(max(p.y >> sb, 0), ny - 1);
  const int cz = D == 3 ? min(max(p.z >> sb, 0), nz - 1) : 0;
  const float oy = (float)(p.y - (cy << sb));
  const float oz = D == 3 ? (float)(p.z - (cz << sb)) : 0.0f;
  const float R2m = (float)I.R2 * (1.0f + 9.5367431640625e-07f);
  const long long base = I.cell_base;
  for (int dz = (D == 3 ? -2 : 0); dz <= (D == 3 ? 2 : 0); ++dz) {
    int z = 0;
    float gz2 = 0.0f;
    if (D == 3) {
      const int zu = cz + dz;
      if (PER && I.period[2]) z = wrap_cell(zu, nz);
      else if (zu < 0 || zu >= nz) continue;
      else z = zu;
      const float gz = fmaxf(slab_gap(dz, oz, S), 0.0f);
      gz2 = gz * gz;
      if (gz2 >= R2m) continue;
    }
    for (int dy = -2; dy <= 2; ++dy) {
      const int yu = cy + dy;
      int y;
      if (PER && I.period[1]) y = wrap_cell(yu, ny);
      else if (yu < 0 || yu >= ny) continue;
      else y = yu;
      const float gy = fmaxf(slab_gap(dy, oy, S), 0.0f);
      const float rem = R2m - gz2 - gy * gy;
      if (rem <= 0.0f) continue;
      // |dx| of a neighbour is below sqrt(rem); rsqrt-based root within 2 quanta
      const long long xr = (long long)(rem * rsqrtf(rem)) + 2;
      int xa = (int)(((long long)p.x - xr) >> sb), xb = (int)(((long long)p.x + xr) >> sb);
      const long long row = base + ((long long)z * ny + y) * nx;
      if (PER && I.period[0]) {
        if (xa < 0) {
          visit(start[row + xa + nx], start[row + nx]);
          xa = 0;
        }
        if (xb >= nx) {
          visit(start[row + xa], start[row + nx]);
          visit(start[row], start[row + xb - nx + 1]);
          continue;
        }
      } else {
        xa = max(xa, 0);
        xb = min(xb, nx - 1);
        if (xa > xb) continue;
      }
      visit(start[row + xa], start[row + xb + 1]);
    }
  }
}

// Appends neighbour indices to one particle's quad-interleaved row (slot s of particle i
// at ((s >> 2) n + i) 4 + (s & 3)) with a running pointer instead of a product per slot.
struct RowWriter {
  int* p;
  int64_t stride;   // 4n ints between consecutive quads of one particle
  int sub, count, cap;
  __device__ __forceinline__ RowWriter(int* nbr, int64_t n, int64_t i, int slot0, int cap_)
      : p(nbr + ((int64_t)(slot0 >> 2) * n + i) * 4), stride(4 * n), sub(slot0 & 3), count(0), cap(cap_ - slot0) {}
  __device__ __forceinline__ void push(int j, bool& overflow) {
    if (count < cap) {
      p[sub] = j;
      if (++sub == 4) {
        sub = 0;
        p += stride;
      }
    } else {
      overflow = true;
    }
    ++count;
  }
};

// Candidate test: the squared distance in FP32 from exactly converted integer
// differences (error < 3 ulp); only inside a +-2^-20 band around the threshold is
// the exact integer test needed, so the decision is always the integer one.
// Two candidates at once in the lanes of packed FP32 instructions. The exact test sits
// behind a warp vote: a warp takes it only when one of its candidates falls in the band
// (measured 0.1 ms faster per build at 8M than selecting between the two tests).
template <int D, bool PER>
__device__ __forceinline__ void within_fast2(const int4& p, const int4& a, const int4& b, const Inst& I,
                                             float lo, float hi, bool& in_a, bool& in_b) {
  const float2 M = f2(-kMagic);
  const float2 dx = add2(make_float2(biased_diff<PER>(p.x, a.x, I.period[0]), biased_diff<PER>(p.x, b.x, I.period[0])), M);
  const float2 dy = add2(make_float2(biased_diff<PER>(p.y, a.y, I.period[1]), biased_diff<PER>(p.y, b.y, I.period[1])), M);
  float2 d2 = fma2(dx, dx, mul2(dy, dy));
  if (D == 3) {
    const float2 dz = add2(make_float2(biased_diff<PER>(p.z, a.z, I.period[2]), biased_diff<PER>(p.z, b.z, I.period[2])), M);
    d2 = fma2(dz, dz, d2);
  }
  in_a = d2.x < lo;
  in_b = d2.y < lo;
  const bool ea = !in_a && d2.x < hi, eb = !in_b && d2.y < hi;
  if (__any_sync(__activemask(), ea || eb)) {
    if (ea) in_a = within<D>(p, a, I);
    if (eb) in_b = within<D>(p, b, I);
  }
}

template <int D, bool PER>
__global__ void __launch_bounds__(kBlock)
k_neighbours(int64_t n, const int4* __restrict__ P, const int* __restrict__ inst_of,
             const Inst* __restrict__ inst, const uint32_t* __restrict__ fstart,
             const int4* __restrict__ WP, const uint32_t* __restrict__ wstart,
             const uint8_t* __restrict__ wnear, int cap, int* __restrict__ nbr,
             uint32_t* __restrict__ nbc, Global* g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = inst[inst_of ? inst_of[i] : 0];
  const float R2f = (float)I.R2;
  const float lo = R2f * (1.0f - 9.5367431640625e-07f), hi = R2f * (1.0f + 9.5367431640625e-07f);
  const int4 pi = P[i];
  bool overflow = false;
  RowWriter fw(nbr, n, i, 0, cap);
  for_neighbour_runs<D, PER>(I, pi, fstart, [&](uint32_t b, uint32_t e) {
    for (uint32_t j = b; j < e; j += 2) {
      const uint32_t j2 = j + 1 < e ? j + 1 : j;     // odd tail: test j twice, keep once
      bool in_a, in_b;
      within_fast2<D, PER>(pi, P[j], P[j2], I, lo, hi, in_a, in_b);
      if (in_a && (int64_t)j != i) fw.push((int)j, overflow);
      if (in_b && j2 != j && (int64_t)j2 != i) fw.push((int)j2, overflow);
    }
  });
  const int nf = min(fw.count, cap);
  int nw = 0;
  if (WP && wnear[search_cell<D>(I, pi)]) {           // no wall within reach: skip the pass
    RowWriter ww(nbr, n, i, wall_slot0(nf), cap);
    for_neighbour_runs<D, PER>(I, pi, wstart, [&](uint32_t b, uint32_t e) {
      for (uint32_t j = b; j < e; j += 2) {
        const uint32_t j2 = j + 1 < e ? j + 1 : j;
        bool in_a, in_b;
        within_fast2<D, PER>(pi, WP[j], WP[j2], I, lo, hi, in_a, in_b);
        if (in_a) ww.push((int)j, overflow);
        if (in_b && j2 != j) ww.push((int)j2, overflow);
      }
    });
    nw = min(ww.count, max(cap - wall_slot0(nf), 0));
  }
  if (overflow) raise_error(g, ERR_CAPACITY, i);
  nbc[i] = (uint32_t)nf | ((uint32_t)nw << 16);
}

// ---------------------------------------------------------------- debug bounds checks --
// SPH_FLAG_DEBUG_BOUNDS: the offsets of a cell-linked list must start at 0, never decrease
// and end at the particle count; a neighbour row must fit the capacity with every fluid
// index below n and every wall index below nw. Each check reads only inside the arrays'
// own extents, whatever values they hold, and records the first violation.
__global__ void k_check_offsets(int64_t n_cells, const uint32_t* __restrict__ start, uint32_t total,
                                Global* g) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > n_cells) return;
  bool bad = start[c] > total;
  if (c == 0) bad = bad || start[0] != 0u;
  if (c == n_cells) bad = bad || start[c] != total;
  else bad = bad || start[c] > start[c + 1];
  if (bad) raise_error(g, ERR_BOUNDS, c);
}

__global__ void k_check_table(int64_t n, int64_t nw, int cap, const int* __restrict__ nbr,
                              const uint32_t* __restrict__ nbc, Global* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t cnt = nbc[i];
  const int nf = (int)(cnt & 0xffffu), nwi = (int)(cnt >> 16);
  if (nf > cap || wall_slot0(nf) + nwi > cap) {
    raise_error(g, ERR_BOUNDS, i);
    return;
  }
  for (int s = 0; s < nf; ++s) {
    const int j = nbr[slot_index(n, i, s)];
    if (j < 0 || (int64_t)j >= n) {
      raise_error(g, ERR_BOUNDS, i);
      return;
    }
  }
  const int w0 = wall_slot0(nf);
  for (int s = 0; s < nwi; ++s) {
    const int w = nbr[slot_index(n, i, w0 + s)];
    if (w < 0 || (int64_t)w >= nw) {
      raise_error(g, ERR_BOUNDS, i);
      return;
    }
  }
}

// ---------------------------------------------------------------- walls ---------------
__global__ void k_wall_reorder(int64_t n, const int* __restrict__ src, const uint32_t* __restrict__ dst,
                               const int* __restrict__ key, const int4* __restrict__ Pin,
                               const float4* __restrict__ Nin, int4* __restrict__ Pout,
                               float4* __restrict__ Nout, int* __restrict__ id_out) {
  int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const int s = src[d];
  const uint32_t t = dst[d];
  Pout[t] = Pin[s];
  Nout[t] = Nin[s];
  id_out[t] = key[d];
}

__global__ void k_iota(int64_t n, int* __restrict__ a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int)i;
}

// Near-wall flags of the search cells: a cell is flagged when a wall particle lies within
// two search cells on every axis, i.e. in the 5^d block the neighbour search visits. The
// occupancy of the wall grid is dilated by +-2 cells one axis at a time.
__device__ __forceinline__ int cell_instance(const Inst* __restrict__ inst, int n_inst, long long c) {
  int lo = 0, hi = n_inst - 1;                 // last instance whose first cell is <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].cell_base <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_wall_occupied(int64_t n_cells, const uint32_t* __restrict__ wstart, uint8_t* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_cells) out[c] = wstart[c + 1] > wstart[c] ? 1 : 0;
}

__global__ void k_dilate_axis(int64_t n_cells, int axis, const Inst* __restrict__ inst, int n_inst,
                              const uint8_t* __restrict__ in, uint8_t* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const Inst& I = inst[cell_instance(inst, n_inst, c)];
  long long stride = 1;
  for (int a = 0; a < axis; ++a) stride *= I.scell[a];
  const int len = I.scell[axis];
  const int pos = (int)(((c - I.cell_base) / stride) % len);
  uint8_t v = 0;
  for (int d = -2; d <= 2; ++d) {
    int p = pos + d;
    if (I.period[axis]) p = p < 0 ? p + len : (p >= len ? p - len : p);
    else if (p < 0 || p >= len) continue;
    v |= in[c + (long long)(p - pos) * stride];
  }
  out[c] = v;
}

// Row pieces of the row-task form (one tank): row r = cy + scell[1] cz holds the search
// cells (0..scell[0]-1, cy, cz), whose particles are contiguous in the cell order.
__global__ void k_row_count(const Inst I, int64_t n_rows, const uint32_t* __restrict__ fstart,
                            uint32_t* __restrict__ cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const long long c0 = I.cell_base + (long long)r * I.scell[0];
  const uint32_t len = fstart[c0 + I.scell[0]] - fstart[c0];
  cnt[r] = (len + 31u) >> 5;
}

__global__ void k_row_fill(const Inst I, int64_t n_rows, const uint32_t* __restrict__ fstart,
                           const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off,
                           int2* __restrict__ task, int64_t cap) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const long long c0 = I.cell_base + (long long)r * I.scell[0];
  const int first = (int)fstart[c0];
  const int len = (int)(fstart[c0 + I.scell[0]] - fstart[c0]);
  const int k_end = (int)cnt[r];
  for (int k = 0; k < k_end; ++k) {
    const int64_t t = (int64_t)off[r] + k;
    if (t >= cap) return;            // not reached: cap >= n/32 + rows bounds the pieces
    task[t] = make_int2(first + 32 * k, min(32, len - 32 * k));
  }
}

}  // namespace

void launch_hash(const Buffers& b, cudaStream_t s, int64_t* launches) {
  cudaMemsetAsync(b.count, 0, sizeof(uint32_t) * b.n_cells, s);
  if (b.n == 0) return;
  if (b.dim == 2)
    k_hash<2><<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.PS, b.inst_of, b.inst, b.cell, b.count, b.rank, b.glob);
  else
    k_hash<3><<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.PS, b.inst_of, b.inst, b.cell, b.count, b.rank, b.glob);
  ++*launches;
}

void launch_fluid_offsets(const Buffers& b, cudaStream_t s, int64_t* launches) {
  scan_exclusive(b.count, b.fstart, b.n_cells, b.scan_tmp, s, launches);
}

void launch_sort_fluid(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.rows_valid) *b.rows_valid = false;     // the row pieces follow the new order
  if (b.n == 0) return;
  k_scatter<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.cell, b.rank, b.fstart, b.id, b.key, b.src);
  // final slots into rank (free after the scatter); sorted ids into cell (free after the rank)
  k_cell_rank<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.cell, b.fstart, b.key, b.src, b.rank);
  int* ids_sorted = reinterpret_cast<int*>(b.cell);
  k_reorder<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.src, b.rank, b.key, b.PS, b.VS, b.PH, b.VH, b.mass,
                                             b.mass_tmp, ids_sorted);
  k_copy_back<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.PH, b.VH, ids_sorted, b.PS, b.VS, b.id, b.mass_tmp,
                                               b.mass);
  *launches += 4;
}

void launch_neighbours(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  const int4* wp = b.nw ? b.WP : nullptr;
  auto kern = b.dim == 2 ? (b.any_periodic ? k_neighbours<2, true> : k_neighbours<2, false>)
                         : (b.any_periodic ? k_neighbours<3, true> : k_neighbours<3, false>);
  kern<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.PS, b.inst_of, b.inst, b.fstart, wp, b.wstart, b.wnear,
                                        b.cap, b.nbr, b.nbc, b.glob);
  ++*launches;
}

void launch_row_tasks(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (!b.row_task || b.n_rows == 0) return;
  const unsigned g = grid_for(b.n_rows);
  k_row_count<<<g, kBlock, 0, s>>>(b.inst0, b.n_rows, b.fstart, b.row_cnt);
  scan_exclusive(b.row_cnt, b.row_off, b.n_rows, b.row_tmp, s, launches);
  k_row_fill<<<g, kBlock, 0, s>>>(b.inst0, b.n_rows, b.fstart, b.row_cnt, b.row_off, b.row_task,
                                  b.row_task_cap);
  *launches += 2;
}

// Walls are static: sort them into cells once. Uses the fluid build scratch
// (cell/rank/count/key/src sized for max(n, nw)); wid_tmp may be b.wid.
void sort_walls(Buffers& b, int4* WP_tmp, float4* WN_tmp, int* wid_tmp, cudaStream_t s) {
  int64_t dummy = 0;
  cudaMemsetAsync(b.count, 0, sizeof(uint32_t) * b.n_cells, s);
  if (b.nw > 0) {
    if (b.dim == 2)
      k_hash<2><<<grid_for(b.nw), kBlock, 0, s>>>(b.nw, b.WP, b.winst_of, b.inst, b.cell, b.count,
                                                  b.rank, b.glob);
    else
      k_hash<3><<<grid_for(b.nw), kBlock, 0, s>>>(b.nw, b.WP, b.winst_of, b.inst, b.cell, b.count,
                                                  b.rank, b.glob);
  }
  scan_exclusive(b.count, b.wstart, b.n_cells, b.scan_tmp, s, &dummy);
  if (b.nw == 0) return;
  k_iota<<<grid_for(b.nw), kBlock, 0, s>>>(b.nw, wid_tmp);
  k_scatter<<<grid_for(b.nw), kBlock, 0, s>>>(b.nw, b.cell, b.rank, b.wstart, wid_tmp, b.key, b.src);
  k_cell_rank<<<grid_for(b.nw), kBlock, 0, s>>>(b.nw, b.cell, b.wstart, b.key, b.src, b.rank);
  int* wids_sorted = reinterpret_cast<int*>(b.cell);
  k_wall_reorder<<<grid_for(b.nw), kBlock, 0, s>>>(b.nw, b.src, b.rank, b.key, b.WP, b.WN, WP_tmp, WN_tmp,
                                                   wids_sorted);
  cudaMemcpyAsync(b.WP, WP_tmp, sizeof(int4) * b.nw, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(b.WN, WN_tmp, sizeof(float4) * b.nw, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(b.wid, wids_sorted, sizeof(int) * b.nw, cudaMemcpyDeviceToDevice, s);
}

void launch_check_offsets(const Buffers& b, cudaStream_t s, int64_t* launches) {
  k_check_offsets<<<grid_for(b.n_cells + 1), kBlock, 0, s>>>(b.n_cells, b.fstart, (uint32_t)b.n, b.glob);
  k_check_offsets<<<grid_for(b.n_cells + 1), kBlock, 0, s>>>(b.n_cells, b.wstart, (uint32_t)b.nw, b.glob);
  *launches += 2;
}

void launch_check_table(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  k_check_table<<<grid_for(b.n), kBlock, 0, s>>>(b.n, b.nw, b.cap, b.nbr, b.nbc, b.glob);
  ++*launches;
}

void launch_iota(int* a, int64_t n, cudaStream_t s) {
  if (n > 0) k_iota<<<grid_for(n), kBlock, 0, s>>>(n, a);
}

// b.wnear from the sorted walls; tmp holds n_cells bytes of scratch.
void flag_near_wall_cells(const Buffers& b, uint8_t* tmp, cudaStream_t s) {
  if (b.n_cells == 0) return;
  const unsigned grid = grid_for(b.n_cells);
  uint8_t* bufs[2] = {b.wnear, tmp};
  k_wall_occupied<<<grid, kBlock, 0, s>>>(b.n_cells, b.wstart, bufs[b.dim & 1]);
  for (int a = 0; a < b.dim; ++a)       // ping-pong so the last pass writes b.wnear
    k_dilate_axis<<<grid, kBlock, 0, s>>>(b.n_cells, a, b.inst, b.n_inst, bufs[(b.dim + a) & 1],
                                          bufs[(b.dim + a + 1) & 1]);
}

}  // namespace sph
