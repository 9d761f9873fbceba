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

// 16-byte copy from global to shared memory that completes asynchronously
// (cp.async); copies are grouped per tile and waited for with
// cp_async_wait<N> (all but the N most recent groups complete).  L1: through
// L1 (the forward gate: the two halves of a 32-byte sector read by different
// warps of a tile come from L2 once), else L2 only (the reverse step, whose
// two gathered states would only evict each other from L1; measured faster).
template <bool L1>
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (L1) asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
  else asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The sector indices of this thread's S slots of one tile (streamed: each
// table entry is read once per gate).
template <int S>
__device__ __forceinline__ void tile_idx(int (&x)[S], const TileMap& tm, int64_t tile) {
  const int* ti = tm.idx + tile * (TILE_T * S);
#pragma unroll
  for (int q = 0; q < S; ++q) x[q] = __ldcs(ti + threadIdx.x + q * TILE_T);
}

// Starts the copies of this thread's slots of one tile into a stage: psi (or,
// STORED, the gate's stored output values, in slot order) and lambda (ADJ).
template <bool ADJ, bool STORED, int S>
__device__ __forceinline__ void tile_fetch(const int (&x)[S], int64_t tile, const cdf* psi, const cdf* lam,
                                           const cdf* store, cdf* sp, cdf* sl) {
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const int slot = threadIdx.x + q * TILE_T;
    if (x[q] < 0) continue;  // unused slot: no block reads it
    cp_async16<!ADJ>(sp + slot, STORED ? store + tile * (TILE_T * S) + slot : psi + x[q]);
    if (ADJ) cp_async16<false>(sl + slot, lam + x[q]);
  }
  cp_async_commit();
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
  cdf* Sbase = reinterpret_cast<cdf*>(smem + tile_head_bytes(t, tm.nreg, tm.nsub, ADJ));
  constexpr int kStage = TILE_T * S * (ADJ ? 2 : 1);  // cdf entries of one stage: psi, then lambda
  const float cpr = (float)t.cp_re, cpi = (float)t.cp_im;
  // The pipeline: tile i is multiplied out of stage i mod NST while the copies
  // of tiles i + 1 .. i + NST - 1 are in flight.  One barrier per tile: after
  // it every thread is done with tile i - 1, whose stage then takes the
  // copies of tile i + NST - 1.
  constexpr int NST = tile_stages(S);
  int64_t tile = t_begin;
  int x0[S], x1[S], x2[S];  // sector indices of the slots of tiles i, i + 1, i + 2
#pragma unroll
  for (int q = 0; q < S; ++q) x0[q] = x1[q] = x2[q] = -1;
  if (tile < t_end) tile_idx<S>(x0, tm, tile);
  if (tile + t_step < t_end) tile_idx<S>(x1, tm, tile + t_step);
  if (NST == 3 && tile + 2 * t_step < t_end) tile_idx<S>(x2, tm, tile + 2 * t_step);
  // The gate's tables, while those table entries are in flight: the block
  // unitaries by asynchronous copy (in the first tile's group), the rest
  // directly; the barrier of the first tile orders them before any use.
  for (int e = threadIdx.x; e < t.nu; e += blockDim.x) cp_async16<true>(Us + e, U + e);
  if (ADJ)
    for (int e = threadIdx.x; e < t.nf; e += blockDim.x) Fs[e] = P.F[t.f_base + e];
  for (int e = threadIdx.x; e < tm.nreg; e += blockDim.x) Rs[e] = tm.reg[e];
  for (int e = threadIdx.x; e < tm.nsub; e += blockDim.x) Ss[e] = tm.sub[e];
  if (tile < t_end) tile_fetch<ADJ, STORED, S>(x0, tile, psi, lam, store, Sbase, Sbase + TILE_T * S);
  else cp_async_commit();
  if (NST == 3) {  // the second tile's copies start before the loop as well
    if (tile + t_step < t_end)
      tile_fetch<ADJ, STORED, S>(x1, tile + t_step, psi, lam, store, Sbase + kStage, Sbase + kStage + TILE_T * S);
    else
      cp_async_commit();
  }
  int stg = 0;
  // Where each of this thread's slots sits in its tile depends only on the
  // region (the tiles of a CTA climb through the regions in order), so it is
  // worked out once per region: the block class c, member a and block k of
  // slot threadIdx.x + q TILE_T, packed as c | a << 6 | k << 10.
  int reg = -1, G = 1;
  int64_t reg_end = -1;
  int dec[S];
  while (tile < t_end) {
    const int64_t ahead = tile + (NST - 1) * t_step, after = ahead + t_step;
    cdf* const Sp = Sbase + stg * kStage;
    cdf* const Sl = Sp + TILE_T * S;
    cp_async_wait<NST - 2>();  // this thread's copies of tile i have landed,
    __syncthreads();           // and every other thread's; tile i - 1 is done
    {
      cdf* const np = Sbase + ((stg + NST - 1) % NST) * kStage;  // tile i - 1's stage
      if (ahead < t_end) tile_fetch<ADJ, STORED, S>(NST == 3 ? x2 : x1, ahead, psi, lam, store, np, np + TILE_T * S);
      else cp_async_commit();  // an empty group keeps one group per tile for the wait above
    }
    int xn[S];
#pragma unroll
    for (int q = 0; q < S; ++q) xn[q] = -1;
    if (after < t_end) tile_idx<S>(xn, tm, after);
    int xs[S];
#pragma unroll
    for (int q = 0; q < S; ++q) xs[q] = x0[q];
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
        const cdf o = make_cdf(acc_get(ar), acc_get(ai));
        psi[x] = o;
        if (store) __stcs(store + tile * (TILE_T * S) + threadIdx.x + q * TILE_T, o);
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
      if (STORED) {  // lambda <- U^dag lambda
        dfacc br, bi;
        acc_zero(br);
        acc_zero(bi);
        for (int l = 0; l < b; ++l) cmac_cb<REALU, true>(br, bi, Ub[l * b + a], Lk[l * G], (a ^ l) & 1);
        lam[x] = make_cdf(acc_get(br), acc_get(bi));
        continue;
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
    stg = (stg + 1) % NST;
    tile += t_step;
  }
  cp_async_wait<0>();  // nothing stays in flight into shared memory past the call
}

}  // namespace cvq
