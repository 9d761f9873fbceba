// k_ham_impl.cuh -- the sector matvec sigma = H psi (Sec. IV.A) over a range
// of sector indices with the fused energy sum Re <psi|sigma>, shared by the
// single-instance kernel and the batched engine.
#pragma once

#include "cvq_internal.cuh"

namespace cvq {

template <int KIND>
__device__ __forceinline__ uint64_t unrank(int64_t x, const SectorDev& S, const int64_t (*G)[DMAX + 1], uint64_t* wR) {
  if (KIND == CVQ_BKC) return bkc_unrank(x, S);
  return bh_unrank(x, S.L, S.N, G, wR);
}

// Index of the tuple w (index x) moved by (dr on mode r, ds on mode s);
// f is the BKC full index, wR the BH suffix sums.
template <int KIND>
__device__ __forceinline__ int64_t moved_index(int64_t x, uint64_t w, uint64_t wR, int64_t f, int r, int dr, int s,
                                               int ds, const SectorDev& S, const int64_t (*G)[DMAX + 1]) {
  if (KIND == CVQ_BKC) {
    int64_t g = f + (int64_t)dr * S.stride[r];
    if (s >= 0) g += (int64_t)ds * S.stride[s];
    return g >> 1;
  } else {
    return x + bh_move_delta(w, wR, r, s, dr, S.L, G);  // number-conserving moves: ds = -dr
  }
}

// Hamiltonian coefficient tables staged in shared memory.
struct HSmem {
  float2 dE[LMAX][DMAX];
  float2 P[4][DMAX][DMAX];
  float2 hop[LMAX], pair[LMAX];
};

// Batched layer kernel, Bose-Hubbard matvec and diagonal-run items: the warp
// walk's tuple buffer follows the item's tables (the Hamiltonian tables, or a
// diagonal run's phase tables) in dynamic shared memory.
__host__ __device__ constexpr size_t batch_walk_offset() {
  return ((sizeof(HSmem) > sizeof(cdf) * (LMAX * DMAX + MAX_RUN_PAIRS * DMAX * DMAX)
               ? sizeof(HSmem)
               : sizeof(cdf) * (LMAX * DMAX + MAX_RUN_PAIRS * DMAX * DMAX)) + 255) & ~(size_t)255;
}
constexpr size_t BATCH_WALK_BYTES = (size_t)NTHREADS / 32 * 32 * WALK_RMAX * sizeof(uint64_t);

__device__ __forceinline__ void load_htabs(HSmem& h, const SectorDev& S) {
  const float2* a = &S.tab->diagE[0][0];
  for (int e = threadIdx.x; e < LMAX * DMAX; e += blockDim.x) (&h.dE[0][0])[e] = a[e];
  const float2* b = &S.tab->P[0][0][0];
  for (int e = threadIdx.x; e < 4 * DMAX * DMAX; e += blockDim.x) (&h.P[0][0][0])[e] = b[e];
  for (int e = threadIdx.x; e < LMAX; e += blockDim.x) {
    h.hop[e] = S.tab->hop[e];
    h.pair[e] = S.tab->pair[e];
  }
}

// Bose-Hubbard hops along a bond (r, r+1) change the rank by an amount that
// depends only on r and the suffix sum R_{r+1} = n_{r+1} + ... + n_{L-1}: the
// rank terms of the positions other than r and r+1 do not change, and at r
// and r+1 the two combinatorial terms that involve n_r and n_{r+1} cancel.
// Dp[r][Q] is the change for x -> x + e_r - e_{r+1} at R_{r+1} = Q; the
// reverse hop x -> x - e_r + e_{r+1} changes the rank by -Dp[r][R_{r+1} + 1].
__device__ __forceinline__ void load_dhop(int32_t (*Dp)[DMAX + 1], const int64_t (*G)[DMAX + 1], const SectorDev& S) {
  for (int e = threadIdx.x; e < LMAX * (DMAX + 1); e += blockDim.x)
    Dp[e / (DMAX + 1)][e % (DMAX + 1)] = (int32_t)bh_hop_delta(G, S.L, S.N, e / (DMAX + 1), e % (DMAX + 1));
}

// sigma[x] = (H psi)[x] at sector index x (occupation tuple w); eacc +=
// Re conj(psi[x]) sigma[x].  Dp (Bose-Hubbard, may be NULL): the hop rank
// changes of load_dhop, used for the bonds (r, r+1).
template <int KIND>
__device__ __forceinline__ void apply_H_one(const SectorDev& S, const int64_t (*Gs)[DMAX + 1],
                                            const int32_t (*Dp)[DMAX + 1], const HSmem& H,
                                            const cdf* __restrict__ psi, cdf* __restrict__ sigma, int64_t x,
                                            uint64_t w, dfacc& eacc) {
  const int L = S.L, Dm1 = S.D - 1;
  const uint64_t wR = (KIND == CVQ_BH) ? bh_suffix(w, L) : 0;
  const int64_t f = (KIND == CVQ_BKC) ? 2 * x + (occ_get(w, L - 1) & 1) : 0;
  const cdf p = psi[x];
  dfacc dg;
  acc_zero(dg);
  for (int r = 0; r < L; ++r) {
    const float2 e = H.dE[r][occ_get(w, r)];
    acc_add(dg, df_make(e.x, e.y));
  }
  const df d = acc_get(dg);
  dfacc ar, ai;
  acc_zero(ar);
  acc_zero(ai);
  acc_mac(ar, d, re_of(p));
  acc_mac(ai, d, im_of(p));
  for (int b = 0; b < S.nb; ++b) {
    const int r = b, s = (b + 1 == L) ? 0 : b + 1;
    const int nr = occ_get(w, r), ns = occ_get(w, s);
    const bool adj = (KIND == CVQ_BH) && Dp && s == r + 1;
    const df h = df_make(H.hop[b].x, H.hop[b].y);
    if (h.h != 0.f) {
      if (ns >= 1 && nr < Dm1) {  // neighbour x + e_r - e_s: sqrt((n_r + 1) n_s)
        const df c = df_mul(h, df_make(H.P[0][nr][ns].x, H.P[0][nr][ns].y));
        const int64_t xn = adj ? x + Dp[r][occ_get(wR, s)] : moved_index<KIND>(x, w, wR, f, r, +1, s, -1, S, Gs);
        const cdf q = psi[xn];
        acc_mac(ar, c, re_of(q));
        acc_mac(ai, c, im_of(q));
      }
      if (nr >= 1 && ns < Dm1) {  // neighbour x - e_r + e_s: sqrt(n_r (n_s + 1))
        const df c = df_mul(h, df_make(H.P[1][nr][ns].x, H.P[1][nr][ns].y));
        const int64_t xn = adj ? x - Dp[r][occ_get(wR, s) + 1] : moved_index<KIND>(x, w, wR, f, r, -1, s, +1, S, Gs);
        const cdf q = psi[xn];
        acc_mac(ar, c, re_of(q));
        acc_mac(ai, c, im_of(q));
      }
    }
    if (KIND == CVQ_BKC) {
      const df pc = df_make(H.pair[b].x, H.pair[b].y);
      if (pc.h != 0.f) {
        if (nr < Dm1 && ns < Dm1) {  // neighbour x + e_r + e_s (a_r a_s lowers it to x)
          const df c = df_mul(pc, df_make(H.P[2][nr][ns].x, H.P[2][nr][ns].y));
          const cdf q = psi[moved_index<KIND>(x, w, wR, f, r, +1, s, +1, S, Gs)];
          acc_mac(ar, c, re_of(q));
          acc_mac(ai, c, im_of(q));
        }
        if (nr >= 1 && ns >= 1) {  // neighbour x - e_r - e_s
          const df c = df_mul(pc, df_make(H.P[3][nr][ns].x, H.P[3][nr][ns].y));
          const cdf q = psi[moved_index<KIND>(x, w, wR, f, r, -1, s, -1, S, Gs)];
          acc_mac(ar, c, re_of(q));
          acc_mac(ai, c, im_of(q));
        }
      }
    }
  }
  const df sr = acc_get(ar), si = acc_get(ai);
  sigma[x] = make_cdf(sr, si);
  acc_mac(eacc, re_of(p), sr);
  acc_mac(eacc, im_of(p), si);
}

// apply_H_one for x = x0, x0 + step, ... < x1, each index unranked on its own.
template <int KIND>
__device__ __forceinline__ void apply_H_range(const SectorDev& S, const int64_t (*Gs)[DMAX + 1], const HSmem& H,
                                              const cdf* __restrict__ psi, cdf* __restrict__ sigma, int64_t x0,
                                              int64_t x1, int64_t step, dfacc& eacc) {
  for (int64_t x = x0; x < x1; x += step) {
    const uint64_t w = unrank<KIND>(x, S, Gs, nullptr);
    apply_H_one<KIND>(S, Gs, nullptr, H, psi, sigma, x, w, eacc);
  }
}

// Pool screen, Eq. (grad): for a generator A = cp G - conj(cp) G^dag whose
// ladder string G moves x by delta (and G^dag by -delta),
//   Re <sigma|A psi> = Re(cp Z_delta) - Re(conj(cp) Z_{-delta}),
//   Z_delta = sum_x F_delta(x) conj(sigma[x]) psi[x + delta],
// with F_delta(x) the ladder factor of the move; for a diagonal generator
// A = i f(n), Re <sigma|A psi> = sum_x f(x) Re(conj(sigma[x]) i psi[x]).
// Every pool element that moves by the same delta (both phases of a beam
// splitter or squeezer, for instance) shares one Z, so one neighbour read
// per distinct shift serves them all.  This accumulates one chunk of at most
// SCREEN_CHUNK shifts (desc[k] = (i, di, j, dj), j < 0 for a single-mode
// move) or diagonal functions (desc[k] = (f type 1..4, i, j, 0)) over
// x = x0, x0 + step, ... < x1: zr, zi hold Re and Im of Z per shift, zr the
// diagonal sums.
template <int KIND>
__device__ __forceinline__ void screen_chunk(const SectorDev& S, const int64_t (*Gs)[DMAX + 1], const float2 (*sq)[5],
                                             bool isdg, const int4* desc, int cnt, const cdf* __restrict__ psi,
                                             const cdf* __restrict__ sigma, int64_t x0, int64_t x1, int64_t step,
                                             dfacc* zr, dfacc* zi) {
  const int L = S.L, Dm1 = S.D - 1;
#pragma unroll
  for (int k = 0; k < SCREEN_CHUNK; ++k) {
    acc_zero(zr[k]);
    acc_zero(zi[k]);
  }
  for (int64_t x = x0; x < x1; x += step) {
    uint64_t wR = 0;
    const uint64_t w = unrank<KIND>(x, S, Gs, &wR);
    const cdf s = sigma[x];
    if (isdg) {
      const cdf p = psi[x];
      dfacc cc;  // Re(conj(s) i p) = s.im p.re - s.re p.im
      acc_zero(cc);
      acc_mac(cc, im_of(s), re_of(p));
      acc_mac(cc, df_neg(re_of(s)), im_of(p));
      const df cv = acc_get(cc);
#pragma unroll
      for (int k = 0; k < SCREEN_CHUNK; ++k) {
        if (k < cnt) {
          const int4 d = desc[k];
          const int ni = occ_get(w, d.y);
          const int f = (d.x == 1) ? ni * ni : (d.x == 2) ? ni * (ni - 1) : (d.x == 3) ? ni : ni * occ_get(w, d.z);
          if (f) acc_macf(zr[k], cv, (float)f);
        }
      }
      continue;
    }
    const int64_t fx = (KIND == CVQ_BKC) ? 2 * x + (occ_get(w, L - 1) & 1) : 0;
#pragma unroll
    for (int k = 0; k < SCREEN_CHUNK; ++k) {
      if (k >= cnt) continue;
      const int4 h = desc[k];  // (i, di, j, dj), j < 0: single mode
      const int ni = occ_get(w, h.x), nj = (h.z >= 0) ? occ_get(w, h.z) : 0;
      if (ni + h.y < 0 || ni + h.y > Dm1 || (h.z >= 0 && (nj + h.w < 0 || nj + h.w > Dm1))) continue;
      df F = df_make(sq[ni][h.y + 2].x, sq[ni][h.y + 2].y);
      if (h.z >= 0) F = df_mul(F, df_make(sq[nj][h.w + 2].x, sq[nj][h.w + 2].y));
      const cdf q = psi[moved_index<KIND>(x, w, wR, fx, h.x, h.y, h.z, h.w, S, Gs)];
      // Z += conj(s) (F q): the ladder factor scales the neighbour first (two
      // df products), then four multiply-accumulates into Z
      const df fr = df_mul(F, re_of(q)), fi = df_mul(F, im_of(q));
      acc_mac(zr[k], re_of(s), fr);
      acc_mac(zr[k], im_of(s), fi);
      acc_mac(zi[k], re_of(s), fi);
      acc_mac(zi[k], df_neg(im_of(s)), fr);
    }
  }
}

}  // namespace cvq
