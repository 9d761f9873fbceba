// k_tile.cu -- tiled block gates: exp(theta A) psi (Sec. IV.B, O_r =
// exp(theta_r A_r)) and the reverse step of the adjoint gradient, reading the
// member indices of every block from a table built once per pool: the table
// build, and the single-gate kernel over every tile of one gate (the tile
// loop itself is in k_tile_impl.cuh, shared with the batched engine).
#include "k_tile_impl.cuh"

namespace cvq {

// ------------------------------------------------------------ table build

// For region blockIdx.y: the sector index of every member of every block of
// every orbit of the region's class.
template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_tile_build(const __grid_constant__ SectorDev S, int i, int j,
                                                         const __grid_constant__ TypeDesc t, PoolDev P,
                                                         const TileRegion* __restrict__ reg,
                                                         const TileSub* __restrict__ subs, int T,
                                                         int* __restrict__ idx, int* __restrict__ bad) {
  __shared__ int64_t G[LMAX][DMAX + 1];
  if (KIND == CVQ_BH) load_G(G, S);
  __syncthreads();
  const TileRegion R = reg[blockIdx.y];
  const int nm = (j >= 0) ? 2 : 1;
  // an index outside the sector would make the gate kernels read and write
  // out of bounds: it is stored as an unused slot and counted instead
  auto put = [&](int64_t pos, int64_t x) {
    if (x >= 0 && x < S.dim) {
      idx[pos] = (int)x;
    } else {
      idx[pos] = -1;
      atomicAdd(bad, 1);
    }
  };
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < R.count; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tpos = (R.tile0 + o / R.G) * T + (o % R.G);
    BkcIdx kx;
    BhIdx hx;
    if (KIND == CVQ_BKC) {
      kx.si = S.stride[i];
      kx.sj = (j >= 0) ? S.stride[j] : 0;
      const int64_t items = bkc_items(S, nm);
      const int64_t tg = (S.L == nm) ? 0 : (int64_t)R.cls * (items / 2) + o;
      int q;
      bkc_orbit(S, i, j, tg, items, kx.f0, q);
    } else {
      hx = bh_idx_of<int64_t>(S, G, i, j, bh_orbit_of_class(S, G, i, j, R.cls, o));
    }
    for (int c = R.sub0; c < R.sub0 + R.nsub; ++c) {
      const TileSub u = subs[c];
      const int2* mem = P.mem + t.mem_base + P.blk[t.blk_base + u.bi].mem_off;
      for (int l = 0; l < u.b; ++l)
        put(tpos + u.off + (int64_t)l * R.G, KIND == CVQ_BKC ? kx(mem[l]) : hx(mem[l]));
    }
  }
}

cudaError_t launch_tile_build(const SectorDev& S, int i, int j, const TypeDesc& t, PoolDev P, const TileRegion* reg_dev,
                              const TileSub* sub_dev, int nreg, int64_t max_count, int tile_slots, int* idx, int* bad,
                              cudaStream_t st) {
  if (nreg <= 0) return cudaSuccess;
  const int64_t want = (max_count + NTHREADS - 1) / NTHREADS;
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 4 * NBLK)), (unsigned)nreg);
  const int T = TILE_T * tile_slots;
  if (S.kind == CVQ_BH) k_tile_build<CVQ_BH><<<grid, NTHREADS, 0, st>>>(S, i, j, t, P, reg_dev, sub_dev, T, idx, bad);
  else k_tile_build<CVQ_BKC><<<grid, NTHREADS, 0, st>>>(S, i, j, t, P, reg_dev, sub_dev, T, idx, bad);
  return cudaGetLastError();
}

// ------------------------------------------------------------ gates

// Resident CTAs per SM of the tiled gates: 5 at one slot per thread; at four,
// 3, except the reverse step that updates both states, which keeps 2 so that
// its larger staging leaves L1 room (measured faster).
__host__ __device__ constexpr int tile_ctas_per_sm(bool adj, int slots, bool stored) {
  return slots == 1 ? 5 : (adj && !stored ? 2 : 3);
}

template <bool ADJ, bool REALU, int S, bool STORED>
__global__ void __launch_bounds__(NTHREADS, tile_ctas_per_sm(ADJ, S, STORED))
    k_tile_gate(const __grid_constant__ GateArg g, PoolDev P, cdf* psi, cdf* lam, cdf* store,
                double* __restrict__ partial) {
  extern __shared__ __align__(16) char smem[];
  dfacc gacc;
  acc_zero(gacc);
  tile_gate_range<ADJ, REALU, S, STORED>(g.t, g.tm, g.U, P, blockIdx.x, g.tm.ntiles, gridDim.x, psi, lam, store, smem,
                                         gacc);
  if (ADJ) {
    const double s = block_sum(acc_to_double(gacc));
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
    if (blockIdx.x == 0)  // the row's slots past the grid hold zeros for the fixed-order reduction
      for (int e = gridDim.x + threadIdx.x; e < NBLK; e += blockDim.x) partial[e] = 0.0;
  }
}

template <bool ADJ, int S, bool STORED>
static cudaError_t launch_tile_impl(const GateArg& g, PoolDev P, cdf* psi, cdf* lam, cdf* store, double* partial,
                                    cudaStream_t st) {
  const size_t sm = tile_smem_bytes(g.t, g.tm.nreg, g.tm.nsub, ADJ, S);
  constexpr int kMaxSmem = 110 * 1024;
  if (sm > (size_t)kMaxSmem) return cudaErrorInvalidValue;
  // one opt-in to the largest dynamic shared memory a gate can need (a
  // function-local static: done once, also when several host threads launch)
  static const bool attr_set = [] {
    cudaFuncSetAttribute(k_tile_gate<ADJ, true, S, STORED>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_tile_gate<ADJ, false, S, STORED>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    return true;
  }();
  (void)attr_set;
  // As many CTAs as fit on the SMs at once, so that no second partial wave
  // runs, and for the forward gate no more than tiles.  The reverse step
  // leaves one partial sum per CTA in its gradient row of NBLK slots (CTAs
  // without a tile write 0, CTA 0 zeroes the slots past the grid), so it
  // takes at most NBLK CTAs.
  const int resident = (NBLK / 4) * tile_ctas_per_sm(ADJ, S, STORED);
  const int grid = ADJ ? std::min(NBLK, resident)
                       : (int)std::max<int64_t>(1, std::min<int64_t>(g.tm.ntiles, resident));
  if (g.t.realu) k_tile_gate<ADJ, true, S, STORED><<<grid, NTHREADS, sm, st>>>(g, P, psi, lam, store, partial);
  else k_tile_gate<ADJ, false, S, STORED><<<grid, NTHREADS, sm, st>>>(g, P, psi, lam, store, partial);
  return cudaGetLastError();
}

cudaError_t launch_tile_gate(const GateArg& g, PoolDev P, cdf* psi, cdf* lam, double* partial, bool adjoint,
                             cudaStream_t st, cdf* store) {
  if (!g.tm.idx || g.t.diag) return cudaErrorInvalidValue;
  if (g.tm.slots == TILE_S_LARGE)
    return adjoint ? launch_tile_impl<true, TILE_S_LARGE, false>(g, P, psi, lam, nullptr, partial, st)
                   : launch_tile_impl<false, TILE_S_LARGE, false>(g, P, psi, nullptr, store, nullptr, st);
  if (g.tm.slots != 1) return cudaErrorInvalidValue;
  return adjoint ? launch_tile_impl<true, 1, false>(g, P, psi, lam, nullptr, partial, st)
                 : launch_tile_impl<false, 1, false>(g, P, psi, nullptr, store, nullptr, st);
}

cudaError_t launch_tile_gate_stored(const GateArg& g, PoolDev P, const cdf* store, cdf* lam, double* partial,
                                    cudaStream_t st) {
  if (!g.tm.idx || g.t.diag || !store) return cudaErrorInvalidValue;
  cdf* sv = const_cast<cdf*>(store);  // read only on this path
  if (g.tm.slots == TILE_S_LARGE) return launch_tile_impl<true, TILE_S_LARGE, true>(g, P, nullptr, lam, sv, partial, st);
  if (g.tm.slots != 1) return cudaErrorInvalidValue;
  return launch_tile_impl<true, 1, true>(g, P, nullptr, lam, sv, partial, st);
}

}  // namespace cvq
