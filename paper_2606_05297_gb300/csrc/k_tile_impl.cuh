// k_tile_impl.cuh -- tiled block gates (Sec. IV.B, O_r = exp(theta_r A_r),
// and the reverse step of the adjoint gradient), shared by the single-gate
// kernel and the batched engine.
//
// A gate acts block-diagonally (the blocks of one orbit are chains of
// occupation pairs joined by the generator's move).  A CTA takes one tile at
// a time: G whole orbits of one class, every block of two or more members of
// them, TILE_T x S table slots.  Each thread loads the S sector indices of its
// slots (coalesced) and the amplitudes they name, the tile is staged in
// shared memory, and each thread then forms the output amplitudes of its
// slots from the staged members of their blocks and the block unitary (also
// in shared memory).  No thread computes a rank, every load of a tile is in
// flight at once, neighbouring amplitudes (whole orbits) are loaded by the
// same tile, and the next tile's loads are issued before the current tile is
// multiplied.  The blocks of one tile are disjoint from every other tile's, so
// the gate runs in place.  Blocks of one member (zero generator: identity) are
// not in the table and are never touched.
#pragma once

#include "cvq_internal.cuh"
#include "k_gate_impl.cuh"

namespace cvq {

// Shared memory of a tiled gate: the gate's block unitaries, the generator
// factors (reverse), the regions, then the staged amplitudes of one tile
// (psi, and lambda in the reverse step).
__host__ __device__ __forceinline__ size_t tile_head_bytes(const TypeDesc& t, int nreg, int nsub, bool adj) {
  size_t b = (size_t)t.nu * sizeof(cdf);
  b += (((size_t)(adj ? t.nf : 0) * sizeof(float2)) + 15) & ~(size_t)15;
  b += (size_t)nreg * sizeof(TileRegion) + (size_t)nsub * sizeof(TileSub);
  return (b + 15) & ~(size_t)15;
}

// Stages of the tile pipeline: while a tile is multiplied out of one stage,
// the copies of the next tiles into the others are in flight: three stages at
// one slot per thread, two at four (whose stages are four times larger).
__host__ __device__ constexpr int tile_stages(int slots) { return slots == 1 ? 3 : 2; }

__host__ __device__ __forceinline__ size_t tile_smem_bytes(const TypeDesc& t, int nreg, int nsub, bool adj, int slots) {
  return tile_head_bytes(t, nreg, nsub, adj) +
         (size_t)tile_stages(slots) * TILE_T * slots * sizeof(cdf) * (adj ? 2 : 1);
}

// 16-byte copy from global to shared memory (address d in the shared state
// space) that completes asynchronously (cp.async); copies are grouped per tile
// and waited for with cp_async_wait<N> (all but the N most recent groups
// complete).  L1: through L1 (the forward gate: the two halves of a 32-byte
// sector read by different warps of a tile come from L2 once), else L2 only
// (the reverse step, whose two gathered states would only evict each other
// from L1; measured faster).
template <bool L1>
__device__ __forceinline__ void cp_async16(unsigned d, const void* gmem_src) {
  if (L1) asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
  else asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The sector indices of this thread's S slots of one tile (streamed: each
// table entry is read once per gate).  Tile and slot offsets are 32-bit: the
// pool build rejects tables of 2^31 or more slots.
template <int S>
__device__ __forceinline__ void tile_idx(int (&x)[S], const int* idx, int tile) {
  const int* ti = idx + (tile * (TILE_T * S) + (int)threadIdx.x);
#pragma unroll
  for (int q = 0; q < S; ++q) x[q] = __ldcs(ti + q * TILE_T);
}

// Starts the copies of this thread's slots of one tile into the stage whose
// slot threadIdx.x is at shared address d: psi (or, STORED, the gate's stored
// output values, in slot order) and lambda (ADJ, TILE_T x S slots further).
template <bool ADJ, bool STORED, int S>
__device__ __forceinline__ void tile_fetch(const int (&x)[S], int tile, const cdf* psi, const cdf* lam,
                                           const cdf* store, unsigned d) {
#pragma unroll
  for (int q = 0; q < S; ++q) {
    if (x[q] < 0) continue;  // unused slot: no block reads it
    const unsigned dq = d + (unsigned)(q * TILE_T * sizeof(cdf));
    cp_async16<!ADJ>(dq, STORED ? store + (tile * (TILE_T * S) + (int)threadIdx.x + q * TILE_T) : psi + x[q]);
    if (ADJ) cp_async16<false>(dq + (unsigned)(TILE_T * S * sizeof(cdf)), lam + x[q]);
  }
  cp_async_commit();
}

// Region of a tile: the last one whose first tile is <= tile.
__device__ __forceinline__ int tile_region(const TileRegion* Rs, int nreg, int tile) {
  int lo = 0, hi = nreg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)Rs[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Where one of a thread's slots sits in the tiles of a region (the same in
// every tile of it): block size b, member a, the staged offset pk of member 0
// of its block (member l at pk + l G), the offset u of the unitary entries it
// reads (forward: row a, entries u + l; reverse: column a, entries u + l b),
// and, reverse, the generator factor F_a of the entries (a, a + 1).
struct TileSlot {
  int b, a, pk, u;
  float fh, fl;
};

// acc += sum over l < b of u[l us] v[l vs] (CONJ: conj(u[l us]) v[l vs]) for a
// row or column of a block unitary whose entry l is real when p + l is even
// and imaginary when it is odd (REALU: every entry real).  The parity is taken
// per entry: warps whose slots mix both parities then stay converged.
template <bool REALU, bool CONJ>
__device__ __forceinline__ void cb_dot(dfacc& ar, dfacc& ai, const cdf* u, int us, const cdf* v, int vs, int b, int p) {
  for (int l = 0; l < b; ++l) cmac_cb<REALU, CONJ>(ar, ai, u[l * us], v[l * vs], (p ^ l) & 1);
}

// Two such sums over the same unitary entries: (ar, ai) over v, (br, bi) over w.
template <bool REALU, bool CONJ>
__device__ __forceinline__ void cb_dot2(dfacc& ar, dfacc& ai, dfacc& br, dfacc& bi, const cdf* u, int us, const cdf* v,
                                        const cdf* w, int vs, int b, int p) {
  for (int l = 0; l < b; ++l) {
    const cdf uu = u[l * us];
    const int odd = (p ^ l) & 1;
    cmac_cb<REALU, CONJ>(ar, ai, uu, v[l * vs], odd);
    cmac_cb<REALU, CONJ>(br, bi, uu, w[l * vs], odd);
  }
}

// Tiles t_begin, t_begin + t_step, ... < t_end of one gate (block unitaries U,
// type t, tiles tm) applied in place to psi (ADJ: the reverse step on psi and
// lambda, its gradient term added to gacc).  Stages the gate's tables in smem
// (tile_smem_bytes of it); the caller synchronises before smem is reused.
// Stored states (forward): when store is not NULL, each output amplitude is
// also written to store in slot order.  STORED (reverse): psi at the gate's
// output is read from store in slot order, the gradient term and lambda <-
// U^dag lambda are formed, and psi itself is neither read nor written.
template <bool ADJ, bool REALU, int S, bool STORED = false>
__device__ __forceinline__ void tile_gate_range(const TypeDesc& t, const TileMap& tm, const cdf* U, const PoolDev& P,
                                                int64_t t_begin, int64_t t_end, int64_t t_step, cdf* psi, cdf* lam,
                                                cdf* store, char* smem, dfacc& gacc) {
  cdf* Us = reinterpret_cast<cdf*>(smem);
  float2* Fs = reinterpret_cast<float2*>(Us + t.nu);
  char* after_f = reinterpret_cast<char*>(Fs) + ((((size_t)(ADJ ? t.nf : 0) * sizeof(float2)) + 15) & ~(size_t)15);
  TileRegion* Rs = reinterpret_cast<TileRegion*>(after_f);
  TileSub* Ss = reinterpret_cast<TileSub*>(Rs + tm.nreg);
  const char* Sbase = smem + tile_head_bytes(t, tm.nreg, tm.nsub, ADJ);
  constexpr int TS = TILE_T * S;                                    // slots of a tile
  constexpr unsigned kStageB = (unsigned)(TS * sizeof(cdf) * (ADJ ? 2 : 1));  // bytes of one stage: psi, then lambda
  const float cpr = (float)t.cp_re, cpi = (float)t.cp_im;
  // The pipeline: tile i is multiplied out of stage i mod NST while the copies
  // of tiles i + 1 .. i + NST - 1 are in flight.  One barrier per tile: after
  // it every thread is done with tile i - 1, whose stage then takes the
  // copies of tile i + NST - 1.
  constexpr int NST = tile_stages(S);
  const int tend = (int)t_end, tstep = (int)t_step;
  int tile = (int)t_begin;
  const unsigned sd = (unsigned)__cvta_generic_to_shared(Sbase) + threadIdx.x * (unsigned)sizeof(cdf);
  int x0[S], x1[S], x2[S];  // sector indices of the slots of tiles i, i + 1, i + 2
#pragma unroll
  for (int q = 0; q < S; ++q) x0[q] = x1[q] = x2[q] = -1;
  if (tile < tend) tile_idx<S>(x0, tm.idx, tile);
  if (tile + tstep < tend) tile_idx<S>(x1, tm.idx, tile + tstep);
  if (NST == 3 && tile + 2 * tstep < tend) tile_idx<S>(x2, tm.idx, tile + 2 * tstep);
  // The gate's tables, while those table entries are in flight: the block
  // unitaries by asynchronous copy (in the first tile's group), the rest
  // directly; the barrier of the first tile orders them before any use.
  {
    const unsigned ud = (unsigned)__cvta_generic_to_shared(Us);
    for (int e = threadIdx.x; e < t.nu; e += blockDim.x) cp_async16<true>(ud + (unsigned)e * sizeof(cdf), U + e);
  }
  if (ADJ)
    for (int e = threadIdx.x; e < t.nf; e += blockDim.x) Fs[e] = P.F[t.f_base + e];
  for (int e = threadIdx.x; e < tm.nreg; e += blockDim.x) Rs[e] = tm.reg[e];
  for (int e = threadIdx.x; e < tm.nsub; e += blockDim.x) Ss[e] = tm.sub[e];
  if (tile < tend) tile_fetch<ADJ, STORED, S>(x0, tile, psi, lam, store, sd);
  else cp_async_commit();
  if (NST == 3) {  // the second tile's copies start before the loop as well
    if (tile + tstep < tend) tile_fetch<ADJ, STORED, S>(x1, tile + tstep, psi, lam, store, sd + kStageB);
    else cp_async_commit();
  }
  unsigned so = 0;  // byte offset of tile i's stage
  // Where each of this thread's slots sits in its tile depends only on the
  // region (the tiles of a CTA climb through the regions in order), so it is
  // worked out once per region.
  int G = 1, reg_end = -1;
  TileSlot ts[S];
  while (tile < tend) {
    const int ahead = tile + (NST - 1) * tstep, after = ahead + tstep;
    const cdf* const Sp = reinterpret_cast<const cdf*>(Sbase + so);
    const cdf* const Sl = Sp + TS;
    cp_async_wait<NST - 2>();  // this thread's copies of tile i have landed,
    __syncthreads();           // and every other thread's; tile i - 1 is done
    {
      const unsigned prev = so == 0 ? (unsigned)(NST - 1) * kStageB : so - kStageB;  // tile i - 1's stage
      if (ahead < tend) tile_fetch<ADJ, STORED, S>(NST == 3 ? x2 : x1, ahead, psi, lam, store, sd + prev);
      else cp_async_commit();  // an empty group keeps one group per tile for the wait above
    }
    int xn[S];
#pragma unroll
    for (int q = 0; q < S; ++q) xn[q] = -1;
    if (after < tend) tile_idx<S>(xn, tm.idx, after);
    int xs[S];
#pragma unroll
    for (int q = 0; q < S; ++q) xs[q] = x0[q];
    if (tile >= reg_end) {
      const int reg = tile_region(Rs, tm.nreg, tile);
      const TileRegion R = Rs[reg];
      G = R.G;
      reg_end = (reg + 1 < tm.nreg) ? (int)Rs[reg + 1].tile0 : (int)tm.ntiles;
#pragma unroll
      for (int q = 0; q < S; ++q) {
        const int slot = threadIdx.x + q * TILE_T;
        int c = R.sub0 + R.nsub - 1;  // the block class whose slots hold this one
        while (c > R.sub0 && Ss[c].off > slot) --c;
        const TileSub u = Ss[c];
        const int rel = slot - u.off;
        const int a = rel / G;
        ts[q].b = u.b;
        ts[q].a = a;
        ts[q].pk = u.off + (rel - a * G);
        ts[q].u = ADJ ? u.u_off + a : u.u_off + a * u.b;
        ts[q].fh = ts[q].fl = 0.f;
        if (ADJ && a + 1 < u.b) {  // a slot past the region's blocks (a >= b) holds -1 in every tile
          const float2 f = Fs[u.f_off + a];
          ts[q].fh = f.x;
          ts[q].fl = f.y;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const int x = xs[q];
      if (x < 0) continue;
      const int b = ts[q].b, a = ts[q].a;
      const cdf* Ub = Us + ts[q].u;
      const cdf* Pk = Sp + ts[q].pk;  // member l of this block at Pk[l * G]
      if (!ADJ) {
        dfacc ar, ai;
        acc_zero(ar);
        acc_zero(ai);
        cb_dot<REALU, false>(ar, ai, Ub, 1, Pk, G, b, a);  // row a of U: entry l imaginary when a + l is odd
        const cdf o = make_cdf(acc_get(ar), acc_get(ai));
        psi[x] = o;
        if (store) __stcs(store + (tile * TS + (int)threadIdx.x + q * TILE_T), o);
        continue;
      }
      const cdf* Lk = Sl + ts[q].pk;
      if (a + 1 < b) {  // gradient term of the generator entries (a, a+1) and (a+1, a)
        const cdf lk = Lk[a * G], lk1 = Lk[(a + 1) * G];
        const cdf pk = Pk[a * G], pk1 = Pk[(a + 1) * G];
        const df Fk = df_make(ts[q].fh, ts[q].fl);
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
      if (STORED) {  // lambda <- U^dag lambda (column a of U, conjugated)
        dfacc br, bi;
        acc_zero(br);
        acc_zero(bi);
        cb_dot<REALU, true>(br, bi, Ub, b, Lk, G, b, a);
        lam[x] = make_cdf(acc_get(br), acc_get(bi));
        continue;
      }
      dfacc ar, ai, br, bi;
      acc_zero(ar);
      acc_zero(ai);
      acc_zero(br);
      acc_zero(bi);
      cb_dot2<REALU, true>(ar, ai, br, bi, Ub, b, Pk, Lk, G, b, a);  // psi <- U^dag psi, lambda <- U^dag lambda
      psi[x] = make_cdf(acc_get(ar), acc_get(ai));
      lam[x] = make_cdf(acc_get(br), acc_get(bi));
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
      x0[q] = x1[q];
      if (NST == 3) {
        x1[q] = x2[q];
        x2[q] = xn[q];
      } else {
        x1[q] = xn[q];
      }
    }
    so = so + kStageB == (unsigned)NST * kStageB ? 0u : so + kStageB;
    tile += tstep;
  }
  cp_async_wait<0>();  // nothing stays in flight into shared memory past the call
}

}  // namespace cvq
