// k_tile.cu -- tiled block gates: exp(theta A) psi (Sec. IV.B, O_r =
// exp(theta_r A_r)) and the reverse step of the adjoint gradient, reading the
// member indices of every block from a table built once per pool.
//
// A gate acts block-diagonally (the blocks of one orbit are chains of
// occupation pairs joined by the generator's move).  Here a CTA takes one
// tile at a time: G whole orbits of one class, every block of two or more
// members of them, TILE_T x S table slots.  Each thread loads the S sector
// indices of its slots (coalesced) and the amplitudes they name, the tile is
// staged in shared memory, and each thread then forms the output amplitudes
// of its slots from the staged members of their blocks and the block
// unitary (also in shared memory).  No thread computes a rank, every load of
// a tile is in flight at once, neighbouring amplitudes (whole orbits) are
// loaded by the same tile, and the next tile's loads are issued before the
// current tile is multiplied.  The blocks of one tile are disjoint from every
// other tile's, so the gate runs in place.  Blocks of one member (zero
// generator: identity) are not in the table and are never touched.
#include "cvq_internal.cuh"
#include "k_gate_impl.cuh"

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

// Shared memory of a tiled gate: the gate's block unitaries, the generator
// factors (reverse), the regions, then the staged amplitudes of one tile
// (psi, and lambda in the reverse step).
__host__ __device__ __forceinline__ size_t tile_head_bytes(const TypeDesc& t, int nreg, int nsub, bool adj) {
  size_t b = (size_t)t.nu * sizeof(cdf);
  b += (((size_t)(adj ? t.nf : 0) * sizeof(float2)) + 15) & ~(size_t)15;
  b += (size_t)nreg * sizeof(TileRegion) + (size_t)nsub * sizeof(TileSub);
  return (b + 15) & ~(size_t)15;
}

__host__ __device__ __forceinline__ size_t tile_smem_bytes(const TypeDesc& t, int nreg, int nsub, bool adj, int slots) {
  return tile_head_bytes(t, nreg, nsub, adj) + (size_t)TILE_T * slots * sizeof(cdf) * (adj ? 2 : 1);
}

// The S slots of one thread in one tile (slot threadIdx.x + q TILE_T), as
// loaded ahead of their multiply.
template <int S>
struct TileSlots {
  int x[S];       // sector index, -1 if the slot is unused
  cdf v[S], l[S]; // psi (and lambda) at x
};

template <bool ADJ, int S>
__device__ __forceinline__ void tile_load(TileSlots<S>& s, const TileMap& tm, int64_t tile, const cdf* psi,
                                          const cdf* lam) {
  const int* ti = tm.idx + tile * (TILE_T * S);
#pragma unroll
  for (int q = 0; q < S; ++q) s.x[q] = __ldcs(ti + threadIdx.x + q * TILE_T);  // streamed once per gate
#pragma unroll
  for (int q = 0; q < S; ++q) {
    s.v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    s.l[q] = s.v[q];
    if (s.x[q] >= 0) {
      s.v[q] = psi[s.x[q]];
      if (ADJ) s.l[q] = lam[s.x[q]];
    }
  }
}

// Region of a tile: the last one whose first tile is <= tile.
__device__ __forceinline__ int tile_region(const TileRegion* Rs, int nreg, int64_t tile) {
  int lo = 0, hi = nreg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (Rs[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <bool ADJ, bool REALU, int S>
__global__ void __launch_bounds__(NTHREADS, S == 1 ? 4 : (S == 2 ? 3 : (ADJ ? 2 : 3))) k_tile_gate(const __grid_constant__ GateArg g, PoolDev P,
                                                                       cdf* psi, cdf* lam,
                                                                       double* __restrict__ partial) {
  extern __shared__ __align__(16) char smem[];
  const TypeDesc& t = g.t;
  const TileMap& tm = g.tm;
  cdf* Us = reinterpret_cast<cdf*>(smem);
  float2* Fs = reinterpret_cast<float2*>(Us + t.nu);
  char* after_f = reinterpret_cast<char*>(Fs) + ((((size_t)(ADJ ? t.nf : 0) * sizeof(float2)) + 15) & ~(size_t)15);
  TileRegion* Rs = reinterpret_cast<TileRegion*>(after_f);
  TileSub* Ss = reinterpret_cast<TileSub*>(Rs + tm.nreg);
  cdf* Sp = reinterpret_cast<cdf*>(smem + tile_head_bytes(t, tm.nreg, tm.nsub, ADJ));
  cdf* Sl = Sp + TILE_T * S;
  for (int e = threadIdx.x; e < t.nu; e += blockDim.x) Us[e] = g.U[e];
  if (ADJ)
    for (int e = threadIdx.x; e < t.nf; e += blockDim.x) Fs[e] = P.F[t.f_base + e];
  for (int e = threadIdx.x; e < tm.nreg; e += blockDim.x) Rs[e] = tm.reg[e];
  for (int e = threadIdx.x; e < tm.nsub; e += blockDim.x) Ss[e] = tm.sub[e];
  __syncthreads();
  const float cpr = (float)t.cp_re, cpi = (float)t.cp_im;
  dfacc gacc;
  acc_zero(gacc);
  int64_t tile = blockIdx.x;
  TileSlots<S> cur;
  if (tile < tm.ntiles) tile_load<ADJ, S>(cur, tm, tile, psi, lam);
  // Where each of this thread's slots sits in its tile depends only on the
  // region (the tiles of a CTA climb through the regions in order), so it is
  // worked out once per region: the block class c, member a and block k of
  // slot threadIdx.x + q TILE_T, packed as c | a << 6 | k << 10.
  int reg = -1, G = 1;
  int64_t reg_end = -1;
  int dec[S];
  while (tile < tm.ntiles) {
    const int64_t next = tile + gridDim.x;
    __syncthreads();  // every thread has finished reading the previous tile
    int xs[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
      Sp[threadIdx.x + q * TILE_T] = cur.v[q];
      if (ADJ) Sl[threadIdx.x + q * TILE_T] = cur.l[q];
      xs[q] = cur.x[q];
    }
    __syncthreads();
    if (next < tm.ntiles) tile_load<ADJ, S>(cur, tm, next, psi, lam);  // in flight during the multiply
    if (tile >= reg_end) {
      reg = tile_region(Rs, tm.nreg, tile);
      const TileRegion R = Rs[reg];
      G = R.G;
      reg_end = (reg + 1 < tm.nreg) ? Rs[reg + 1].tile0 : tm.ntiles;
#pragma unroll
      for (int q = 0; q < S; ++q) {
        const int slot = threadIdx.x + q * TILE_T;
        int c = R.sub0 + R.nsub - 1;  // the block class whose slots hold this one
        while (c > R.sub0 && Ss[c].off > slot) --c;
        const int rel = slot - Ss[c].off;
        const int a = rel / G;
        dec[q] = c | (a << 6) | ((rel - a * G) << 10);
      }
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const int x = xs[q];
      if (x < 0) continue;
      const int c = dec[q] & 63, a = (dec[q] >> 6) & 15, k = dec[q] >> 10;
      const TileSub u = Ss[c];
      const int b = u.b;
      const cdf* Ub = Us + u.u_off;
      const cdf* Pk = Sp + u.off + k;  // member l of this block at Pk[l * G]
      if (!ADJ) {
        dfacc ar, ai;
        acc_zero(ar);
        acc_zero(ai);
        for (int l = 0; l < b; ++l) cmac_cb<REALU, false>(ar, ai, Ub[a * b + l], Pk[l * G], (a ^ l) & 1);
        psi[x] = make_cdf(acc_get(ar), acc_get(ai));
        continue;
      }
      const cdf* Lk = Sl + u.off + k;
      if (a + 1 < b) {  // gradient term of the generator entries (a, a+1) and (a+1, a)
        const cdf lk = Lk[a * G], lk1 = Lk[(a + 1) * G];
        const cdf pk = Pk[a * G], pk1 = Pk[(a + 1) * G];
        const df Fk = df_make(Fs[u.f_off + a].x, Fs[u.f_off + a].y);
        if (cpr != 0.f) {  // Re z_a
          dfacc z;
          acc_zero(z);
          acc_mac(z, re_of(lk), re_of(pk1));
          acc_mac(z, im_of(lk), im_of(pk1));
          acc_mac(z, df_neg(re_of(lk1)), re_of(pk));
          acc_mac(z, df_neg(im_of(lk1)), im_of(pk));
          const df zr = acc_get(z);
          acc_mac(gacc, Fk, df_make(zr.h * cpr, zr.l * cpr));
        }
        if (cpi != 0.f) {  // -Im z_a
          dfacc z;
          acc_zero(z);
          acc_mac(z, re_of(lk), im_of(pk1));
          acc_mac(z, df_neg(im_of(lk)), re_of(pk1));
          acc_mac(z, df_neg(im_of(lk1)), re_of(pk));
          acc_mac(z, re_of(lk1), im_of(pk));
          const df zi = acc_get(z);
          acc_mac(gacc, Fk, df_make(-zi.h * cpi, -zi.l * cpi));
        }
      }
      dfacc ar, ai, br, bi;
      acc_zero(ar);
      acc_zero(ai);
      acc_zero(br);
      acc_zero(bi);
      for (int l = 0; l < b; ++l) {  // psi <- U^dag psi, lambda <- U^dag lambda
        const cdf uu = Ub[l * b + a];
        const int odd = (a ^ l) & 1;
        cmac_cb<REALU, true>(ar, ai, uu, Pk[l * G], odd);
        cmac_cb<REALU, true>(br, bi, uu, Lk[l * G], odd);
      }
      psi[x] = make_cdf(acc_get(ar), acc_get(ai));
      lam[x] = make_cdf(acc_get(br), acc_get(bi));
    }
    tile = next;
  }
  if (ADJ) {
    const double s = block_sum(acc_to_double(gacc));
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

template <bool ADJ, int S>
static cudaError_t launch_tile_impl(const GateArg& g, PoolDev P, cdf* psi, cdf* lam, double* partial, cudaStream_t st) {
  const size_t sm = tile_smem_bytes(g.t, g.tm.nreg, g.tm.nsub, ADJ, S);
  constexpr int kMaxSmem = 110 * 1024;
  if (sm > (size_t)kMaxSmem) return cudaErrorInvalidValue;
  static bool attr_set = false;  // one opt-in to the largest dynamic shared memory a gate can need
  if (!attr_set) {
    cudaFuncSetAttribute(k_tile_gate<ADJ, true, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_tile_gate<ADJ, false, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    attr_set = true;
  }
  // The reverse step leaves one partial sum per CTA in each of the NBLK slots
  // of its gradient row (CTAs without a tile write 0); the forward gate needs
  // no more CTAs than tiles.
  const int grid = ADJ ? NBLK : (int)std::max<int64_t>(1, std::min<int64_t>(g.tm.ntiles, NBLK));
  if (g.t.realu) k_tile_gate<ADJ, true, S><<<grid, NTHREADS, sm, st>>>(g, P, psi, lam, partial);
  else k_tile_gate<ADJ, false, S><<<grid, NTHREADS, sm, st>>>(g, P, psi, lam, partial);
  return cudaGetLastError();
}

cudaError_t launch_tile_gate(const GateArg& g, PoolDev P, cdf* psi, cdf* lam, double* partial, bool adjoint,
                             cudaStream_t st) {
  if (!g.tm.idx || g.t.diag) return cudaErrorInvalidValue;
  if (g.tm.slots == TILE_S_LARGE)
    return adjoint ? launch_tile_impl<true, TILE_S_LARGE>(g, P, psi, lam, partial, st)
                   : launch_tile_impl<false, TILE_S_LARGE>(g, P, psi, nullptr, nullptr, st);
  if (g.tm.slots == TILE_S_MID)
    return adjoint ? launch_tile_impl<true, TILE_S_MID>(g, P, psi, lam, partial, st)
                   : launch_tile_impl<false, TILE_S_MID>(g, P, psi, nullptr, nullptr, st);
  if (g.tm.slots != 1) return cudaErrorInvalidValue;
  return adjoint ? launch_tile_impl<true, 1>(g, P, psi, lam, partial, st)
                 : launch_tile_impl<false, 1>(g, P, psi, nullptr, nullptr, st);
}

}  // namespace cvq
