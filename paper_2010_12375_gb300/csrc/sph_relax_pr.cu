// Pressure relaxation launches (kernels and pair terms in sph_relax.cuh) and the
// frozen-geometry table. Its own translation unit so the two relaxation kernels compile
// in parallel.
#include "sph_relax.cuh"

namespace sph {

namespace {

// Frozen-geometry reading: the pair vector r_i - r_j and (dW/dr)/r of every neighbour slot
// at the configuration update, with the same operations the relaxation kernels use on
// positions (zero half-step shift), into geo[slot][n]. Pad slots of a partial quad hold
// the particle itself (r = 0) for fluid quads and the quad's first wall for wall quads,
// as the relaxation kernels pad them.
template <int D, bool PER, bool UNI>
__global__ void __launch_bounds__(128)
k_pair_geometry(const Inst Ip, int64_t n, const int4* __restrict__ PS, const int* __restrict__ inst_of,
                const Inst* __restrict__ inst, const int* __restrict__ nbr, const uint32_t* __restrict__ nbc,
                const int4* __restrict__ WP, float4* __restrict__ geo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst& I = UNI ? Ip : inst[inst_index(inst_of, i)];
  const int4 pi = PS[i];
  const uint32_t cnt = nbc[i];
  const int nf = (int)(cnt & 0xffffu), nw = (int)(cnt >> 16);
  const int px = PER ? I.period[0] : 0, py = PER ? I.period[1] : 0, pz = PER ? I.period[2] : 0;
  const float2 DQ = f2(I.dq), Z = f2(0.f);
  const int4* __restrict__ nb4 = reinterpret_cast<const int4*>(nbr);
  auto store = [&](int64_t slot0, const int4& a, const int4& b) {
    const float2 rx = pair_axis<PER>(pi.x, a.x, b.x, px, DQ, Z);
    const float2 ry = pair_axis<PER>(pi.y, a.y, b.y, py, DQ, Z);
    float2 rz = Z;
    if (D == 3) rz = pair_axis<PER>(pi.z, a.z, b.z, pz, DQ, Z);
    const Geo2 G = geometry2(rx, ry, rz, I.inv_h, I.dwr_a);
    geo[slot0 * n + i] = make_float4(rx.x, ry.x, rz.x, G.fw.x);
    geo[(slot0 + 1) * n + i] = make_float4(rx.y, ry.y, rz.y, G.fw.y);
  };
  const int nq = (nf + 3) >> 2;
  for (int q = 0; q < nq; ++q) {
    const int4 c = nb4[(int64_t)q * n + i];
    const int s = q << 2;
    const int j1 = s + 1 < nf ? c.y : (int)i, j2 = s + 2 < nf ? c.z : (int)i, j3 = s + 3 < nf ? c.w : (int)i;
    store(s, PS[c.x], PS[j1]);
    store(s + 2, PS[j2], PS[j3]);
  }
  if (nw) {
    const int q0 = wall_slot0(nf) >> 2, nwq = (nw + 3) >> 2;
    for (int q = 0; q < nwq; ++q) {
      const int4 c = nb4[(int64_t)(q0 + q) * n + i];
      const int s = q << 2;
      const int w1 = s + 1 < nw ? c.y : c.x, w2 = s + 2 < nw ? c.z : c.x, w3 = s + 3 < nw ? c.w : c.x;
      store((q0 + q) << 2, WP[c.x], WP[w1]);
      store(((q0 + q) << 2) + 2, WP[w2], WP[w3]);
    }
  }
}

template <int D, bool PER>
void launch_geo(const Buffers& b, cudaStream_t s) {
  const unsigned grid = grid_for(b.n, 128);
  const int4* wp = b.nw ? b.WP : nullptr;
  if (b.n_inst == 1)
    k_pair_geometry<D, PER, true><<<grid, 128, 0, s>>>(b.inst0, b.n, b.PS, b.inst_of, b.inst, b.nbr, b.nbc, wp, b.geo);
  else
    k_pair_geometry<D, PER, false><<<grid, 128, 0, s>>>(b.inst0, b.n, b.PS, b.inst_of, b.inst, b.nbr, b.nbc, wp, b.geo);
}

}  // namespace

void launch_pair_geometry(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0 || !b.geo) return;
  if (b.dim == 2) {
    if (b.any_periodic) launch_geo<2, true>(b, s);
    else launch_geo<2, false>(b, s);
  } else {
    if (b.any_periodic) launch_geo<3, true>(b, s);
    else launch_geo<3, false>(b, s);
  }
  ++*launches;
}

void launch_pressure_relaxation(const Buffers& b, cudaStream_t s, int64_t* launches) {
  if (b.n == 0) return;
  const int tpp = b.cfg.pr_tpp;
  int block = b.cfg.pr_block;
  if (row_form(block)) {
    if (!b.row_task || b.geo) {
      block = 128;                        // row pieces exist for one tank only
    } else if (!*b.rows_valid) {           // first row-task launch since the cells changed
      launch_row_tasks(b, s, launches);
      *b.rows_valid = true;
    }
  }
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
