// k_diag_impl.cuh -- runs of consecutive diagonal gates (K, R, CK, n(n-1);
// they commute) applied over a range of sector indices as one phase
// multiply, forward or as the fused reverse step of the adjoint gradient.
// Shared by the single-instance kernel and the batched engine.
#pragma once

#include "cvq_internal.cuh"

namespace cvq {

// complex df multiply-accumulate helpers for the diagonal runs
__device__ __forceinline__ void cmac_full(dfacc& ar, dfacc& ai, cdf u, cdf v) {  // += u v
  acc_mac(ar, re_of(u), re_of(v));
  acc_mac(ai, re_of(u), im_of(v));
  acc_mac(ar, df_neg(im_of(u)), im_of(v));
  acc_mac(ai, im_of(u), re_of(v));
}

__device__ __forceinline__ void cmac_conj_full(dfacc& ar, dfacc& ai, cdf u, cdf v) {  // += conj(u) v
  acc_mac(ar, re_of(u), re_of(v));
  acc_mac(ai, re_of(u), im_of(v));
  acc_mac(ar, im_of(u), im_of(v));
  acc_mac(ai, df_neg(im_of(u)), re_of(v));
}

// psi[x] *= prod_r T[r][n_r] * prod_p TP[p][n_i D + n_j] at sector index x
// (occupation tuple w), the first product over the modes a single-mode gate of
// the run acts on (T is 1 on every other mode, and at n_r = 0).  A carries the
// run's gate list (m, npair, diag, gi, gj, pi, pj) and its modes (nact, act).
// ADJ: acc[k] += Re(conj(lam) i f_k psi) at the run's output state, then psi
// and lam are multiplied by the conjugate phase (KEEP: psi, read from dst, is
// the stored output state and is left as it is; only lam is multiplied).
template <bool ADJ, int NACC, class A, bool KEEP = false>
__device__ __forceinline__ void diag_run_one(const SectorDev& S, const cdf (*T)[DMAX], const cdf (*TP)[DMAX * DMAX],
                                             const A& a, const cdf* src, cdf* dst, cdf* lam, int64_t x, uint64_t w,
                                             dfacc (&acc)[NACC]) {
  const int D = S.D;
  df pr = df_make(1.f, 0.f), pi = df_make(0.f, 0.f);
  for (int q = 0; q < a.nact; ++q) {
    const int r = a.act[q];
    const int n = occ_get(w, r);
    if (n == 0) continue;
    const cdf t = T[r][n];
    const df nr = df_add(df_mul(pr, re_of(t)), df_neg(df_mul(pi, im_of(t))));
    const df ni = df_add(df_mul(pr, im_of(t)), df_mul(pi, re_of(t)));
    pr = nr;
    pi = ni;
  }
  for (int p = 0; p < a.npair; ++p) {
    const int v = occ_get(w, a.pi[p]) * D + occ_get(w, a.pj[p]);
    const cdf t = TP[p][v];
    const df nr = df_add(df_mul(pr, re_of(t)), df_neg(df_mul(pi, im_of(t))));
    const df ni = df_add(df_mul(pr, im_of(t)), df_mul(pi, re_of(t)));
    pr = nr;
    pi = ni;
  }
  if (!ADJ) {
    const cdf v = src[x];
    dfacc ar, ai;
    acc_zero(ar);
    acc_zero(ai);
    cmac_full(ar, ai, make_cdf(pr, pi), v);
    dst[x] = make_cdf(acc_get(ar), acc_get(ai));
  } else {
    const cdf ps = dst[x], la = lam[x];
    // Re(conj(la) * i f ps) = f * (la.im ps.re - la.re ps.im)
    dfacc c;
    acc_zero(c);
    acc_mac(c, im_of(la), re_of(ps));
    acc_mac(c, df_neg(re_of(la)), im_of(ps));
    const df cv = acc_get(c);
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
      if (k < a.m) {
        const int ni = occ_get(w, a.gi[k]);
        const int dg = a.diag[k];
        const int f = (dg == 1) ? ni * ni : (dg == 2) ? ni * (ni - 1) : (dg == 3) ? ni : ni * occ_get(w, a.gj[k]);
        if (f) acc_macf(acc[k], cv, (float)f);
      }
    }
    const cdf ph = make_cdf(pr, pi);
    dfacc r1, i1, r2, i2;
    acc_zero(r1);
    acc_zero(i1);
    acc_zero(r2);
    acc_zero(i2);
    if (!KEEP) {
      cmac_conj_full(r1, i1, ph, ps);
      dst[x] = make_cdf(acc_get(r1), acc_get(i1));
    }
    cmac_conj_full(r2, i2, ph, la);
    lam[x] = make_cdf(acc_get(r2), acc_get(i2));
  }
}

// diag_run_one for x = x0, x0 + step, ... < x1, each index unranked on its own.
template <int KIND, bool ADJ, int NACC, class A>
__device__ __forceinline__ void diag_run_range(const SectorDev& S, const int64_t (*Gs)[DMAX + 1],
                                               const cdf (*T)[DMAX], const cdf (*TP)[DMAX * DMAX], const A& a,
                                               const cdf* src, cdf* dst, cdf* lam, int64_t x0, int64_t x1,
                                               int64_t step, dfacc (&acc)[NACC]) {
  for (int64_t x = x0; x < x1; x += step) {
    const uint64_t w = (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, S.L, S.N, Gs);
    diag_run_one<ADJ, NACC>(S, T, TP, a, src, dst, lam, x, w, acc);
  }
}

// Gradient terms only, at a run's output state, for gates beyond the
// accumulators of the reverse pass: acc[k] += Re(conj(lam) i f_k psi) at
// sector index x (tuple w), no table, no write.
template <int NACC, class A>
__device__ __forceinline__ void diag_grad_one(const A& a, const cdf* __restrict__ psi, const cdf* __restrict__ lam,
                                              int64_t x, uint64_t w, dfacc (&acc)[NACC]) {
  const cdf ps = psi[x], la = lam[x];
  dfacc c;
  acc_zero(c);
  acc_mac(c, im_of(la), re_of(ps));
  acc_mac(c, df_neg(re_of(la)), im_of(ps));
  const df cv = acc_get(c);
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
    if (k < a.m) {
      const int ni = occ_get(w, a.gi[k]);
      const int dg = a.diag[k];
      const int f = (dg == 1) ? ni * ni : (dg == 2) ? ni * (ni - 1) : (dg == 3) ? ni : ni * occ_get(w, a.gj[k]);
      if (f) acc_macf(acc[k], cv, (float)f);
    }
  }
}

// diag_grad_one for x = x0, x0 + step, ... < x1.
template <int KIND, int NACC, class A>
__device__ __forceinline__ void diag_grad_range(const SectorDev& S, const int64_t (*Gs)[DMAX + 1], const A& a,
                                                const cdf* __restrict__ psi, const cdf* __restrict__ lam, int64_t x0,
                                                int64_t x1, int64_t step, dfacc (&acc)[NACC]) {
  for (int64_t x = x0; x < x1; x += step) {
    const uint64_t w = (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, S.L, S.N, Gs);
    diag_grad_one<NACC>(a, psi, lam, x, w, acc);
  }
}

}  // namespace cvq
